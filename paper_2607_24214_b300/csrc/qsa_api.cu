// C ABI of the QS-PIC hot path (declarations and contracts in include/qsa.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <atomic>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qsa.h"
#include <nvtx3/nvToolsExt.h>
#include "qsa_beam.cuh"
#include "qsa_common.cuh"
#include "qsa_fft.cuh"
#include "qsa_pipe.cuh"
#include "qsa_sweep.cuh"
#include "qsa_tables.h"
#include "qsa_adjoint.cuh"
#include "qsa_rehome.cuh"

using namespace qsa;

namespace {

thread_local std::string g_init_error;

constexpr int kThreads = 256;

bool size_ok(int n) {
  if (n < 1 || n > QSA_MAX_N) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

struct Base {
  virtual ~Base() {}
};

}  // namespace

struct qsa_handle {
  qsa_params prm;
  cudaStream_t stream = nullptr;
  qsa_alloc_fn alloc = nullptr;
  qsa_free_fn free_fn = nullptr;
  void* ctx = nullptr;
  int num_sms = 0;
  DevParams dp{};
  std::vector<std::pair<void*, size_t>> allocs;
  int64_t bytes = 0;
  int64_t launches = 0;
  int64_t sweeps = 0;
  int64_t pushes = 0;  // beam pushes done: the source and extent rings are indexed by it
  bool src_valid = false;
  std::string err;
  // typed state lives behind these pointers (R = double for FP64, float for mixed)
  bool fp64 = true;
  void* st = nullptr;
  // CUDA events around the persistent launches of the last pipelined qsa_advance
  static constexpr int kLaunchEvents = 64;
  cudaEvent_t ev[2 * kLaunchEvents] = {};
  int n_timed = 0;
  // the run recorded by qsa_grad_forward for qsa_grad_backward (null: none)
  struct GradRun* grad = nullptr;
  bool beam_replaced = false;  // qsa_set_beam replaced the beam qsa_init built
  int64_t rehomes = 0;         // re-homings of the beam done (qsa_rehome, qsa_advance)
  int last_pushes = 0;         // pushes of the last pipelined launch
  uint64_t serial = 0;         // unique over the process's handles, never reused
  // CUDA graphs of the batched steps this handle leads (qsa_advance_batch)
  std::vector<struct BatchGraph*> graphs;
  bool batch_graphs = true;    // capture and replay the batched steps
  bool graphs_failed = false;  // a capture failed: launch directly from then on
  int64_t graph_replays = 0;
  cudaStream_t cap_stream = nullptr;  // the stream the batched steps are captured on
};

// One batched step as a CUDA graph: the same stream work for the same handles, FFT unit
// shape and ring phases (every pointer the step touches is fixed by them).  The slot tables
// it uploads live in pinned host memory of its own.
struct BatchGraph {
  std::vector<uint64_t> serials;
  std::vector<int64_t> phases;
  int nbr = 0, nbc = 0;
  int ev_end = 0;  // the launch events it records: the lead's ev[0 .. 2 ev_end) at most
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> tables;
  ~BatchGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    for (void* t : tables) cudaFreeHost(t);
  }
};

// State of a differentiable run between qsa_grad_forward and qsa_grad_backward.
struct GradRun {
  int n_steps = 0, ckpt = 10;
  double loss = 0.0;
  std::vector<double*> beam_ckpt;  // beam state after 0, ckpt, 2 ckpt, ... pushes
  double* beam_end = nullptr;      // beam state after n_steps pushes
  int64_t pushes = 0, sweeps = 0;  // the handle's counters after the forward run
};

namespace {

}  // namespace

namespace qsa {
// Message for qsa_last_error(NULL) from entry points that have no handle.
void set_global_error(const std::string& msg) { g_init_error = msg; }
int static_bounds_counts(unsigned long long* first, unsigned long long* count);
}  // namespace qsa

namespace {

int fail(qsa_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_init_error = msg;
  return code;
}

int cuda_fail(qsa_handle* h, cudaError_t e, const char* what) {
  return fail(h, QSA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void* dalloc(qsa_handle* h, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (h->alloc) {
    p = h->alloc(bytes, h->ctx, (void*)h->stream);
  } else if (cudaMallocAsync(&p, bytes, h->stream) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    h->allocs.push_back({p, bytes});
    h->bytes += (int64_t)bytes;
  }
  return p;
}

// Release one allocation made through dalloc.
void dfree(qsa_handle* h, void* p) {
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i].first == p) {
      const auto a = h->allocs[i];
      h->allocs.erase(h->allocs.begin() + (long)i);
      h->bytes -= (int64_t)a.second;
      if (h->free_fn) h->free_fn(a.first, a.second, h->ctx, (void*)h->stream);
      else cudaFreeAsync(a.first, h->stream);
      return;
    }
}

void dfree_all(qsa_handle* h) {
  for (auto& a : h->allocs) {
    if (h->free_fn) h->free_fn(a.first, a.second, h->ctx, (void*)h->stream);
    else cudaFreeAsync(a.first, h->stream);
  }
  h->allocs.clear();
}

template <typename R>
struct State {
  using BR = R;
  // sweep slots: slot 0 serves the single sweep; a pipelined launch of m steps uses 0..m-1
  std::vector<SweepArgs<R>> slots;
  int last_slot = 0;                // slot of the last sweep (slab, diagnostics)
  std::vector<BeamArrays<BR>> beams;
  std::vector<SpeciesDev> species;
  std::vector<BeamConst<R>> bconst;
  ModesDev modes{};
  std::vector<R*> srcs;             // source ring, S + 1 entries [nk][ny][nx][4]
  std::vector<int*> cmaxs;          // extent ring, S + 1 entries [nxi]
  std::vector<double*> moms;        // beam-moment ring, S + 1 entries [n_species][nxi][7]
  int* dmin = nullptr;              // min over live particles of (xi cell - home layer)
  int* chk = nullptr;               // set by check_xi_kernel when a host beam is invalid
  PipeTable<R>* ptab = nullptr;     // device table of the multi-slot launches (lazy)
  int tuned_nbr = 0, tuned_nbc = 0; // FFT units chosen by the batch autotuner (0: not yet)
  unsigned long long* lost = nullptr;
  unsigned long long* away = nullptr;  // beam particles outside their slots' cells (pipelined)
  // re-homing buffers (lazy): cell keys of a chunk of layers, per-cell counts, prefix sums and
  // cursors, per-layer cursors of the lost particles, and staging arrays of the chunk
  int rh_layers = 0;
  int *rh_key = nullptr, *rh_cnt = nullptr, *rh_exc = nullptr, *rh_vac = nullptr,
      *rh_cur = nullptr, *rh_dead = nullptr;
  BeamArrays<R> rh_t{};
  unsigned* bar = nullptr;  // [0] count, [1] generation
  int* status = nullptr;
  C<R>* tw = nullptr;
  double* bref = nullptr;          // [nk] beam J_z reference density per node (device)
  unsigned long long* ptimes = nullptr;  // phase timestamps of the first slices
  R* ktab = nullptr;                     // wavenumber table of the k-space solves
  std::vector<double> bref_s, bref_jz;  // host copies of the S_b and J_z references
  size_t smem = 0;
  int grid = 0;
};

template <typename R>
State<R>* S(qsa_handle* h) { return reinterpret_cast<State<R>*>(h->st); }

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);    \
  } while (0)

// Ring entries of the beam state after `pushes` pushes: its sources and its extents.
template <typename R>
R* ring_src(qsa_handle* h, int64_t pushes) {
  State<R>* s = S<R>(h);
  return s->srcs[(size_t)(pushes % (int64_t)s->srcs.size())];
}
template <typename R>
int* ring_cmax(qsa_handle* h, int64_t pushes) {
  State<R>* s = S<R>(h);
  return s->cmaxs[(size_t)(pushes % (int64_t)s->cmaxs.size())];
}
template <typename R>
double* ring_mom(qsa_handle* h, int64_t pushes) {
  State<R>* s = S<R>(h);
  return s->moms[(size_t)(pushes % (int64_t)s->moms.size())];
}
size_t mom_bytes(const qsa_handle* h) {
  const int ns = h->prm.n_species > 0 ? h->prm.n_species : 1;
  return (size_t)ns * (h->dp.nxi > 0 ? h->dp.nxi : 1) * 7 * sizeof(double);
}
// Zero the extent and moment ring entries that the beam state after `pushes` pushes fills.
template <typename R>
int clear_ring(qsa_handle* h, int64_t pushes) {
  CK(cudaMemsetAsync(ring_cmax<R>(h, pushes), 0xFF,
                     (size_t)(h->dp.nxi > 0 ? h->dp.nxi : 1) * sizeof(int), h->stream));
  CK(cudaMemsetAsync(ring_mom<R>(h, pushes), 0, mom_bytes(h), h->stream));
  return QSA_OK;
}


template <typename R>
size_t sweep_smem(const DevParams& dp) {
  return sweep_smem_bytes<R>(dp.nx, dp.ny);
}

template <typename R>
int setup(qsa_handle* h) {
  State<R>* s = new State<R>();
  h->st = s;
  const DevParams& dp = h->dp;
  const size_t g = (size_t)dp.nx * dp.ny;
  const size_t spec = (size_t)dp.nxh * dp.ny;
  auto A = [&](size_t bytes) { return dalloc(h, bytes); };
  const int nslot = h->prm.pipeline_depth > 1 ? h->prm.pipeline_depth : 1;  // depth S
  // tables shared by every slot
  R* ktab = (R*)A((size_t)(2 * dp.nxh + 2 * dp.ny) * sizeof(R));
  C<R>* twp = (C<R>*)A((size_t)(dp.nx + dp.ny) * sizeof(C<R>));
  double* bref = (double*)A((size_t)dp.nk * sizeof(double));
  unsigned* bar = (unsigned*)A(2 * sizeof(unsigned));
  int* status = (int*)A(sizeof(int));
  s->lost = (unsigned long long*)A(sizeof(unsigned long long));
  s->away = (unsigned long long*)A(sizeof(unsigned long long));
  s->dmin = (int*)A(sizeof(int));
  s->chk = (int*)A(sizeof(int));
  if (!ktab || !twp || !bref || !bar || !status || !s->lost || !s->dmin || !s->chk || !s->away)
    return fail(h, QSA_ERR_OOM, "sweep tables");
  {
    const std::vector<R> kt = wavenumber_table<R>(dp.nx, dp.ny, dp.Lx, dp.Ly);
    CK(cudaMemcpyAsync(ktab, kt.data(), kt.size() * sizeof(R), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  {
    const std::vector<C<R>> tw = twiddle_table<R>(dp.nx, dp.ny);
    CK(cudaMemcpyAsync(twp, tw.data(), tw.size() * sizeof(C<R>), cudaMemcpyHostToDevice,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  CK(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), h->stream));
  CK(cudaMemsetAsync(status, 0, sizeof(int), h->stream));
  CK(cudaMemsetAsync(s->lost, 0, sizeof(unsigned long long), h->stream));
  CK(cudaMemsetAsync(s->dmin, 0, sizeof(int), h->stream));
  // launch shapes of the persistent kernels
  const size_t smem = sweep_smem<R>(dp);
  CK(raise_dyn_smem((const void*)sweep_kernel<R>, smem));
  CK(raise_dyn_smem((const void*)solve_kernel<R>, smem));
  CK(raise_dyn_smem((const void*)beam_kernel<R, false>, beam_smem_bytes<R>(dp.nx)));
  CK(raise_dyn_smem((const void*)beam_kernel<R, true>, beam_smem_bytes<R>(dp.nx)));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<R>, kThreads, smem));
  int per_sm2 = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, solve_kernel<R>, kThreads, smem));
  per_sm = per_sm < per_sm2 ? per_sm : per_sm2;
  if (per_sm < 1) return fail(h, QSA_ERR_ARG, "sweep kernel does not fit on an SM");
  const int work = dp.ny > dp.nxh ? dp.ny : dp.nxh;
  int grid = per_sm * h->num_sms;
  if (grid > work) grid = work;
  // blocks whose diagnostic partials a slot holds: the single sweep's grid, or a multi-slot
  // launch's (its register budget allows kPipeBlocksPerSM resident blocks per SM at most)
  int dgrid = grid;
  if (kPipeBlocksPerSM * h->num_sms > dgrid) dgrid = kPipeBlocksPerSM * h->num_sms;
  // sweep slots
  s->slots.resize(nslot);
  for (int i = 0; i < nslot; ++i) {
    SweepArgs<R>& a = s->slots[i];
    a = SweepArgs<R>{};
    a.p = dp;
    a.k = sweep_consts<R>(dp);
    const size_t np = (size_t)dp.np;
    R** pl[5] = {&a.pox, &a.poy, &a.pux, &a.puy, &a.ppsi};
    for (auto q : pl) if (!(*q = (R*)A(np * sizeof(R)))) return fail(h, QSA_ERR_OOM, "plasma");
    if (!(a.fg = (R*)A(g * kFG * sizeof(R))) ||
        !(a.part = (R*)A((size_t)dp.ny * kTileRows * dp.nx * kNF * sizeof(R))) ||
        !(a.ovf = (R*)A(g * kNF * sizeof(R))) ||
        !(a.cflag = (int*)A((size_t)dp.ny * sizeof(int))) ||
        !(a.odirty = (int*)A((size_t)dp.ny * sizeof(int))) ||
        !(a.rspec = (C<R>*)A(kNF * spec * sizeof(C<R>))) ||
        !(a.cspec = (C<R>*)A(4 * spec * sizeof(C<R>))) ||
        !(a.jprev = (C<R>*)A(2 * spec * sizeof(C<R>))) ||
        !(a.bold = (C<R>*)A(2 * spec * sizeof(C<R>))) ||
        !(a.slab = (R*)A((size_t)dp.nk * g * 8 * sizeof(R))) ||
        !(a.diag = (double*)A((size_t)D_COUNT * dp.nk * sizeof(double))) ||
        !(a.dpart = (double*)A((size_t)dp.nk * dgrid * P_COUNT * sizeof(double))))
      return fail(h, QSA_ERR_OOM, "sweep buffers");
    if (i == 0 &&
        !(a.ptimes = (unsigned long long*)A(kTimedSlices * kTimedPhases * 2 * 8)))
      return fail(h, QSA_ERR_OOM, "sweep buffers");
    if (dp.nmodes > 0 &&
        !(a.mode_out = (R*)A((size_t)dp.nk * dp.nmodes * 10 * sizeof(R))))
      return fail(h, QSA_ERR_OOM, "mode buffers");
    a.twx = twp;
    a.twy = twp + dp.nx;
    a.ktab = ktab;
    a.bref = bref;
    a.src = nullptr;
    a.bar = Barrier{bar, status, (long long)h->prm.spin_limit};
    CK(cudaMemsetAsync(a.slab, 0, (size_t)dp.nk * g * 8 * sizeof(R), h->stream));
    CK(cudaMemsetAsync(a.diag, 0, (size_t)D_COUNT * dp.nk * sizeof(double), h->stream));
    CK(cudaMemsetAsync(a.cflag, 0, (size_t)dp.ny * sizeof(int), h->stream));
    CK(cudaMemsetAsync(a.odirty, 0, (size_t)dp.ny * sizeof(int), h->stream));
  }
  s->grid = grid;
  s->smem = smem;
  // source and extent rings
  for (int i = 0; i <= nslot; ++i) {
    R* sb = (R*)A((size_t)dp.nk * g * 4 * sizeof(R));
    int* cm = (int*)A((size_t)(dp.nxi > 0 ? dp.nxi : 1) * sizeof(int));
    double* mo = (double*)A(mom_bytes(h));
    if (!sb || !cm || !mo) return fail(h, QSA_ERR_OOM, "source ring");
    s->srcs.push_back(sb);
    s->cmaxs.push_back(cm);
    s->moms.push_back(mo);
  }
  // beam species
  const qsa_params& P = h->prm;
  s->modes.n = P.n_modes;
  for (int m = 0; m < P.n_modes; ++m) {
    s->modes.mx[m] = P.modes[m].mx;
    s->modes.my[m] = P.modes[m].my;
    s->modes.amp[m] = P.modes[m].amplitude;
    s->modes.phase[m] = P.modes[m].phase;
  }
  for (int si = 0; si < P.n_species; ++si) {
    const qsa_species& q = P.species[si];
    SpeciesDev sp{};
    sp.Z = q.Z; sp.M = q.M; sp.alpha = q.alpha; sp.gamma_b = q.gamma_b;
    sp.gamma_spread_rel = q.gamma_spread_rel; sp.uperp_spread = q.uperp_spread;
    sp.noise_rel = q.noise_rel;
    sp.ppx = q.ppc_x; sp.ppy = q.ppc_y; sp.ppxi = q.ppc_xi;
    sp.ppc = q.ppc_x * q.ppc_y * q.ppc_xi;
    const double back = q.xi_back < 0 ? P.Lxi : q.xi_back;
    sp.k0 = (int)std::lround(q.xi_front / dp.dxi);
    sp.nkb = (int)std::lround(back / dp.dxi) - sp.k0;
    sp.seeded = q.seeded;
    sp.index = si;
    sp.wbar = q.alpha * dp.dx * dp.dy * dp.dxi / sp.ppc;
    sp.qbar = q.Z * q.alpha / sp.ppc;
    {
      const double uzb = std::sqrt(q.gamma_b * q.gamma_b - 1.0);
      sp.omvbar = 1.0 / (q.gamma_b * (q.gamma_b + uzb));
      sp.uzb = uzb;
    }
    BeamArrays<R> b{};
    b.n = (long long)dp.nx * dp.ny * sp.nkb * sp.ppc;
    const size_t n = (size_t)b.n;
    if (!(b.ox = (R*)A(n * sizeof(R))) || !(b.oy = (R*)A(n * sizeof(R))) ||
        !(b.oxi = (R*)A(n * sizeof(R))) || !(b.ux = (R*)A(n * sizeof(R))) ||
        !(b.uy = (R*)A(n * sizeof(R))) || !(b.dw = (R*)A(n * sizeof(R))) ||
        !(b.uz = (typename UzT<R>::T*)A(n * sizeof(typename UzT<R>::T))))
      return fail(h, QSA_ERR_OOM, "beam arrays");  // the ids come with the first re-homing
    s->species.push_back(sp);
    s->bconst.push_back(beam_consts<R>(dp, sp));
    s->beams.push_back(b);
    if (b.n > 0) {
      const unsigned blocks = (unsigned)((b.n + kThreads - 1) / kThreads);
      beam_init_kernel<R><<<blocks, kThreads, 0, h->stream>>>(b, dp, sp, s->modes, P.seed);
      ++h->launches;
      CK(cudaGetLastError());
    }
  }
  // uniform reference of the beam sources per node (k = 0 only): Z alpha (1 - v_z) and
  // Z alpha v_z of the reference momentum, times the lattice fill of the node (1 inside the
  // beam, 1/2 on its first and last node)
  s->bref_s.assign(dp.nk, 0.0);
  s->bref_jz.assign(dp.nk, 0.0);
  for (size_t si = 0; si < s->species.size(); ++si) {
    const SpeciesDev& sp = s->species[si];
    if (sp.nkb < 1) continue;
    for (int k = sp.k0; k <= sp.k0 + sp.nkb && k < dp.nk; ++k) {
      const double e = (k == sp.k0 || k == sp.k0 + sp.nkb) ? 0.5 : 1.0;
      const double rho = sp.Z * P.species[si].alpha * e;
      s->bref_s[k] += rho * sp.omvbar;
      s->bref_jz[k] += rho * (1.0 - sp.omvbar);
    }
  }
  CK(cudaMemcpyAsync(bref, s->bref_jz.data(), dp.nk * sizeof(double), cudaMemcpyHostToDevice,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return QSA_OK;
}

template <typename R>
int deposit_sources(qsa_handle* h) {
  State<R>* s = S<R>(h);
  const DevParams& dp = h->dp;
  R* src = ring_src<R>(h, h->pushes);
  int* cmax = ring_cmax<R>(h, h->pushes);
  double* mom = ring_mom<R>(h, h->pushes);
  CK(cudaMemsetAsync(src, 0, (size_t)dp.nk * dp.nx * dp.ny * 4 * sizeof(R), h->stream));
  if (int rc = clear_ring<R>(h, h->pushes)) return rc;
  CK(cudaMemsetAsync(s->dmin, 0, sizeof(int), h->stream));
  for (size_t si = 0; si < s->beams.size(); ++si) {
    const auto& b = s->beams[si];
    if (b.n == 0) continue;
    const unsigned groups = (unsigned)(s->species[si].nkb * dp.ny);
    beam_kernel<R, false><<<groups, kThreads, beam_smem_bytes<R>(dp.nx), h->stream>>>(
        b, dp, s->species[si], s->bconst[si], nullptr, src, nullptr,
        Extent{cmax, s->dmin, mom + si * (size_t)dp.nxi * 7, nullptr});
    ++h->launches;
    CK(cudaGetLastError());
  }
  h->src_valid = true;
  return QSA_OK;
}

__global__ void diag_init_kernel(double* diag, int nk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < D_COUNT * nk) diag[i] = 0.0;
}

// Reduce the per-block partial diagnostics of each slice (one block per slice).
__global__ void diag_reduce_kernel(const double* dpart, int nblk, double* diag, int nk) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  const double* row = dpart + (size_t)j * nblk * P_COUNT;
  for (int f = 0; f < P_COUNT; ++f) {
    double v = (f == P_OPPMIN) ? 1e300 : 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      const double x = row[(size_t)b * P_COUNT + f];
      if (f == P_OPPMIN) v = fmin(v, x);
      else if (f == P_INV) v = fmax(v, x);
      else v += x;
    }
    double r;
    if (f == P_OPPMIN) r = block_min(v, red);
    else if (f == P_INV) r = block_max(v, red);
    else r = block_sum(v, red);
    if (threadIdx.x == 0) {
      int d;
      switch (f) {
        case P_OPPMIN: d = D_OPPMIN; break;
        case P_NFLOOR: d = D_NFLOOR; break;
        case P_INV: d = D_INV; break;
        case P_CHARGE: d = D_CHARGE; break;
        case P_PCNUM: d = D_PCNUM; break;
        case P_PCDEN: d = D_PCDEN; break;
        default: d = D_E0 + (f - P_E0); break;
      }
      diag[(size_t)d * nk + j] = r;
    }
  }
}

template <typename R>
int sweep(qsa_handle* h) {
  State<R>* s = S<R>(h);
  const DevParams& dp = h->dp;
  if (!h->src_valid) {
    int rc = deposit_sources<R>(h);
    if (rc) return rc;
  }
  const size_t g = (size_t)dp.nx * dp.ny;
  const size_t spec = (size_t)dp.nxh * dp.ny;
  SweepArgs<R>& a = s->slots[0];
  CK(cudaMemsetAsync(a.ovf, 0, g * kNF * sizeof(R), h->stream));
  CK(cudaMemsetAsync(a.odirty, 0, (size_t)dp.ny * sizeof(int), h->stream));
  CK(cudaMemsetAsync(a.bold, 0, 2 * spec * sizeof(C<R>), h->stream));
  CK(cudaMemsetAsync(a.fg, 0, g * kFG * sizeof(R), h->stream));
  CK(cudaMemsetAsync(a.bar.count, 0, sizeof(unsigned), h->stream));
  CK(cudaMemsetAsync(a.ptimes, 0, kTimedSlices * kTimedPhases * 2 * 8, h->stream));
  const int nd = D_COUNT * dp.nk;
  diag_init_kernel<<<(nd + 255) / 256, 256, 0, h->stream>>>(a.diag, dp.nk);
  ++h->launches;
  a.src = ring_src<R>(h, h->pushes);
  void* args[] = {&a};
  CK(cudaLaunchCooperativeKernel((void*)sweep_kernel<R>, dim3(s->grid), dim3(kThreads), args,
                                 s->smem, h->stream));
  ++h->launches;
  diag_reduce_kernel<<<dp.nk, 256, 0, h->stream>>>(a.dpart, s->grid, a.diag, dp.nk);
  ++h->launches;
  ++h->sweeps;
  s->last_slot = 0;
  return QSA_OK;
}

// ---- multi-slot launches (chained steps of one handle, or one step of several handles)

// The beam side of a slot whose beam state has had `pushes` pushes.
template <typename R>
PipeSlot<R> make_slot(qsa_handle* h, int64_t pushes) {
  State<R>* s = S<R>(h);
  PipeSlot<R> ps{};
  ps.src_next = ring_src<R>(h, pushes + 1);
  ps.cmax_in = ring_cmax<R>(h, pushes);
  ps.cmax_out = ring_cmax<R>(h, pushes + 1);
  ps.mom_out = ring_mom<R>(h, pushes + 1);
  ps.dmin = s->dmin;
  ps.lost = s->lost;
  ps.away = s->away;
  ps.nspecies = (int)s->species.size();
  for (int si = 0; si < ps.nspecies; ++si) {
    ps.beam[si] = s->beams[si];
    ps.sp[si] = s->species[si];
    ps.bc[si] = s->bconst[si];
  }
  return ps;
}

// Zero what slot `a` of handle h starts from: the next sources and ring entries, the sweep
// scratch that must start at zero, the diagnostics.
template <typename R>
int prepare_slot(qsa_handle* h, SweepArgs<R>& a, int64_t pushes) {
  const DevParams& dp = h->dp;
  const size_t g = (size_t)dp.nx * dp.ny, spec = (size_t)dp.nxh * dp.ny;
  CK(cudaMemsetAsync(ring_src<R>(h, pushes + 1), 0, (size_t)dp.nk * g * 4 * sizeof(R),
                     h->stream));
  if (int rc = clear_ring<R>(h, pushes + 1)) return rc;
  CK(cudaMemsetAsync(a.ovf, 0, g * kNF * sizeof(R), h->stream));
  CK(cudaMemsetAsync(a.odirty, 0, (size_t)dp.ny * sizeof(int), h->stream));
  CK(cudaMemsetAsync(a.bold, 0, 2 * spec * sizeof(C<R>), h->stream));
  CK(cudaMemsetAsync(a.fg, 0, g * kFG * sizeof(R), h->stream));
  const int nd = D_COUNT * dp.nk;
  diag_init_kernel<<<(nd + 255) / 256, 256, 0, h->stream>>>(a.diag, dp.nk);
  ++h->launches;
  return QSA_OK;
}

// Upload table t (nslots slots, FFT units nbr x nbc) to the lead handle's device table and
// launch the multi-slot kernel on the lead's stream, timed with the lead's events.  Returns
// the grid in *grid_out (the diagnostic partials of every slot span it).
template <typename R>
int launch_slots(qsa_handle* lead, PipeTable<R>& t, int nslots, int nbr, int nbc,
                 int* grid_out) {
  qsa_handle* h = lead;
  State<R>* s = S<R>(h);
  t.nbr = nbr;
  t.nbc = nbc;
  t.max_push = 2;
  t.nx_max = t.ny_max = 1;
  for (int i = 0; i < nslots; ++i) {
    t.nx_max = std::max(t.nx_max, t.st[i].p.nx);
    t.ny_max = std::max(t.ny_max, t.st[i].p.ny);
  }
  const size_t smem = pipe_smem_bytes<R>(t.nx_max, t.ny_max, nbr, nbc);
  CK(raise_dyn_smem((const void*)pipe_kernel<R>, smem));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pipe_kernel<R>, kThreads, smem));
  if (per_sm < 1) return fail(h, QSA_ERR_ARG, "multi-slot kernel does not fit on an SM");
  int grid = std::min(per_sm, kPipeBlocksPerSM) * h->num_sms;
  if (!h->ev[0])
    for (int i = 0; i < 2 * qsa_handle::kLaunchEvents; ++i) CK(cudaEventCreate(&h->ev[i]));
  if (!s->ptab && !(s->ptab = (PipeTable<R>*)dalloc(h, sizeof(PipeTable<R>))))
    return fail(h, QSA_ERR_OOM, "slot table");
  // pageable source: the call returns once t is staged, so t may change right after
  CK(cudaMemcpyAsync(s->ptab, &t, sizeof(PipeTable<R>), cudaMemcpyHostToDevice, h->stream));
  Barrier bar = s->slots[0].bar;
  CK(cudaMemsetAsync(bar.count, 0, sizeof(unsigned), h->stream));
  const int ti = h->n_timed < qsa_handle::kLaunchEvents ? h->n_timed++ : -1;
  // under stream capture (a batched step becoming a CUDA graph) the events become event-record
  // nodes of the graph, re-recorded at every replay
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(h->stream, &cap));
  const unsigned evf = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
  if (ti >= 0) CK(cudaEventRecordWithFlags(h->ev[2 * ti], h->stream, evf));
  const PipeTable<R>* tab = s->ptab;
  void* args[] = {&tab, &nslots, &bar};
  CK(cudaLaunchCooperativeKernel((void*)pipe_kernel<R>, dim3(grid), dim3(kThreads), args, smem,
                                 h->stream));
  ++h->launches;
  if (ti >= 0) CK(cudaEventRecordWithFlags(h->ev[2 * ti + 1], h->stream, evf));
  *grid_out = grid;
  return QSA_OK;
}

// FFT units of the chained launches: grid rows and half-spectrum columns per unit (build
// settings for tuning)
#ifndef QSA_PIPE_ROW_BATCH
#define QSA_PIPE_ROW_BATCH 2
#endif
#ifndef QSA_PIPE_COL_BATCH
#define QSA_PIPE_COL_BATCH 1
#endif
constexpr int kPipeRowBatch = QSA_PIPE_ROW_BATCH, kPipeColBatch = QSA_PIPE_COL_BATCH;

// Re-home every species' beam (see qsa_rehome.cuh), a chunk of xi layers at a time.
template <typename R>
int rehome(qsa_handle* h) {
  State<R>* s = S<R>(h);
  const DevParams& dp = h->dp;
  const int ncell = dp.nx * dp.ny;
  int ppc_max = 1, nkb_max = 1;
  for (const auto& sp : s->species) {
    ppc_max = std::max(ppc_max, sp.ppc);
    nkb_max = std::max(nkb_max, sp.nkb);
  }
  const size_t L = (size_t)ncell * ppc_max;
  const size_t rec = 6 * sizeof(R) + sizeof(typename UzT<R>::T) + sizeof(unsigned) + sizeof(int);
  if (!s->rh_layers) {
    // staging of about 1 GB (at least one layer)
    const int nl = (int)std::max<size_t>(1, std::min<size_t>(nkb_max, (size_t(1) << 30) / (L * rec)));
    auto A = [&](size_t bytes) { return dalloc(h, bytes); };
    BeamArrays<R>& t = s->rh_t;
    const size_t m = (size_t)nl * L;
    if (!(s->rh_key = (int*)A(m * sizeof(int))) ||
        !(s->rh_cnt = (int*)A((size_t)nl * ncell * sizeof(int))) ||
        !(s->rh_exc = (int*)A((size_t)nl * ncell * sizeof(int))) ||
        !(s->rh_vac = (int*)A((size_t)nl * ncell * sizeof(int))) ||
        !(s->rh_cur = (int*)A((size_t)nl * ncell * sizeof(int))) ||
        !(s->rh_dead = (int*)A((size_t)nl * sizeof(int))) || !(t.ox = (R*)A(m * sizeof(R))) ||
        !(t.oy = (R*)A(m * sizeof(R))) || !(t.oxi = (R*)A(m * sizeof(R))) ||
        !(t.ux = (R*)A(m * sizeof(R))) || !(t.uy = (R*)A(m * sizeof(R))) ||
        !(t.dw = (R*)A(m * sizeof(R))) ||
        !(t.uz = (typename UzT<R>::T*)A(m * sizeof(typename UzT<R>::T))) ||
        !(t.id = (unsigned*)A(m * sizeof(unsigned))))
      return fail(h, QSA_ERR_OOM, "re-homing buffers");
    s->rh_layers = nl;
  }
  for (size_t si = 0; si < s->beams.size(); ++si) {
    BeamArrays<R>& b = s->beams[si];
    const SpeciesDev& sp = s->species[si];
    if (b.n == 0) continue;
    if (!b.id) {  // every slot holds its own particle until now
      if (!(b.id = (unsigned*)dalloc(h, (size_t)b.n * sizeof(unsigned))))
        return fail(h, QSA_ERR_OOM, "beam ids");
      const unsigned blocks = (unsigned)((b.n + kThreads - 1) / kThreads);
      beam_id_init_kernel<R><<<blocks, kThreads, 0, h->stream>>>(b, dp, sp);
      ++h->launches;
      CK(cudaGetLastError());
    }
    const long long Ls = (long long)ncell * sp.ppc;
    for (int k0 = 0; k0 < sp.nkb; k0 += s->rh_layers) {
      const int nl = std::min(s->rh_layers, sp.nkb - k0);
      const long long m = (long long)nl * Ls;
      const unsigned blocks = (unsigned)((m + kThreads - 1) / kThreads);
      CK(cudaMemsetAsync(s->rh_cnt, 0, (size_t)nl * ncell * sizeof(int), h->stream));
      CK(cudaMemsetAsync(s->rh_dead, 0, (size_t)nl * sizeof(int), h->stream));
      rehome_count_kernel<R><<<blocks, kThreads, 0, h->stream>>>(b, dp, sp, k0, nl, s->rh_key,
                                                                  s->rh_cnt);
      rehome_scan_kernel<<<nl, kRehomeThreads, 0, h->stream>>>(dp, sp.ppc, s->rh_cnt, s->rh_exc,
                                                               s->rh_vac, s->rh_cur);
      rehome_scatter_kernel<R><<<blocks, kThreads, 0, h->stream>>>(
          b, s->rh_t, dp, sp, k0, nl, s->rh_key, s->rh_cnt, s->rh_exc, s->rh_vac, s->rh_cur,
          s->rh_dead);
      h->launches += 3;
      CK(cudaGetLastError());
      const size_t off = (size_t)k0 * Ls;
      const BeamArrays<R>& t = s->rh_t;
      CK(cudaMemcpyAsync(b.ox + off, t.ox, m * sizeof(R), cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(b.oy + off, t.oy, m * sizeof(R), cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(b.oxi + off, t.oxi, m * sizeof(R), cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(b.ux + off, t.ux, m * sizeof(R), cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(b.uy + off, t.uy, m * sizeof(R), cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(b.dw + off, t.dw, m * sizeof(R), cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(b.uz + off, t.uz, m * sizeof(typename UzT<R>::T),
                         cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(b.id + off, t.id, m * sizeof(unsigned), cudaMemcpyDeviceToDevice,
                         h->stream));
    }
  }
  ++h->rehomes;
  h->last_pushes = 0;  // the away count no longer describes the beam
  return QSA_OK;
}

// n beam steps (sweep + push each) as wavefronts of up to S steps per persistent launch.
template <typename R>
int advance_pipelined(qsa_handle* h, int n) {
  State<R>* s = S<R>(h);
  const DevParams& dp = h->dp;
  const int nslot = (int)s->slots.size();
  if (!h->src_valid) {
    int rc = deposit_sources<R>(h);
    if (rc) return rc;
  }
  std::vector<PipeTable<R>> tv(1);  // ~30 KB: on the heap
  PipeTable<R>& t = tv[0];
  int64_t nbeam = 0;
  for (const auto& b : s->beams) nbeam += b.n;
  while (n > 0) {
    const int m = n < nslot ? n : nslot;
    // the away counter holds the pushes of the last pipelined launch (last_pushes of them)
    if (h->last_pushes > 0 && h->prm.rehome_frac > 0.0 && nbeam > 0) {
      unsigned long long away = 0;
      CK(cudaMemcpyAsync(&away, s->away, sizeof(away), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      // each of the last launch's pushes counted its particles that left their slots' cells
      if ((double)away > h->prm.rehome_frac * (double)nbeam * h->last_pushes)
        if (int rc = rehome<R>(h)) return rc;
    }
    CK(cudaMemsetAsync(s->away, 0, sizeof(unsigned long long), h->stream));
    h->last_pushes = m;
    t = PipeTable<R>{};
    t.chained = 1;
    for (int i = 0; i < m; ++i) {
      if (int rc = prepare_slot<R>(h, s->slots[i], h->pushes + i)) return rc;
      t.st[i] = s->slots[i];
      t.st[i].src = ring_src<R>(h, h->pushes + i);
      t.slot[i] = make_slot<R>(h, h->pushes + i);
      // only the last step's beam moments are ever read (qsa_diagnostics reports the state
      // after the last push); the away count only feeds re-homing
      if (i + 1 < m) t.slot[i].mom_out = nullptr;
      if (!(h->prm.rehome_frac > 0.0)) t.slot[i].away = nullptr;
    }
    int grid = 0;
    if (int rc = launch_slots<R>(h, t, m, kPipeRowBatch, kPipeColBatch, &grid)) return rc;
    for (int i = 0; i < m; ++i) {
      SweepArgs<R>& a = s->slots[i];
      diag_reduce_kernel<<<dp.nk, 256, 0, h->stream>>>(a.dpart, grid, a.diag, dp.nk);
      ++h->launches;
    }
    h->pushes += m;
    h->sweeps += m;
    s->last_slot = m - 1;
    n -= m;
  }
  h->src_valid = true;
  return QSA_OK;
}

// FFT unit shapes the batch autotuner tries (rows x half-spectrum columns per unit).
constexpr int kTuneShapes[4][2] = {{2, 1}, {1, 1}, {4, 1}, {2, 2}};

// The stream work of one batched step (every handle by one step, kMaxPipe per launch): slot
// preparation, the launches and the diagnostic reductions, for the handles' current push
// counts; tables[c] (one per launch) holds the slot table the launch uploads.  The host-side
// counters are advanced by finish_batch_step.
template <typename R>
int issue_batch_step(qsa_handle* const* hs, int nh, int nbr, int nbc,
                     PipeTable<R>* const* tables, int* failed) {
  qsa_handle* lead = hs[0];
  for (int c0 = 0, c = 0; c0 < nh; c0 += kMaxPipe, ++c) {
    const int m = std::min(kMaxPipe, nh - c0);
    PipeTable<R>& t = *tables[c];
    t = PipeTable<R>{};
    t.chained = 0;
    for (int i = 0; i < m; ++i) {
      qsa_handle* h = hs[c0 + i];
      SweepArgs<R>& a = S<R>(h)->slots[0];
      if (int rc = prepare_slot<R>(h, a, h->pushes)) {
        *failed = c0 + i;
        return rc;
      }
      t.st[i] = a;
      t.st[i].src = ring_src<R>(h, h->pushes);
      t.slot[i] = make_slot<R>(h, h->pushes);
    }
    int grid = 0;
    if (int rc = launch_slots<R>(lead, t, m, nbr, nbc, &grid)) {
      *failed = 0;
      return rc;
    }
    for (int i = 0; i < m; ++i) {
      qsa_handle* h = hs[c0 + i];
      SweepArgs<R>& a = S<R>(h)->slots[0];
      diag_reduce_kernel<<<h->dp.nk, 256, 0, h->stream>>>(a.dpart, grid, a.diag, h->dp.nk);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        *failed = c0 + i;
        return cuda_fail(h, e, "diag_reduce_kernel");
      }
    }
  }
  return QSA_OK;
}

template <typename R>
void finish_batch_step(qsa_handle* const* hs, int nh) {
  for (int i = 0; i < nh; ++i) {
    qsa_handle* h = hs[i];
    h->launches += 2;  // the diagnostic initialisation and reduction
    h->pushes += 1;
    h->sweeps += 1;
    S<R>(h)->last_slot = 0;
    h->src_valid = true;
  }
  hs[0]->launches += (nh + kMaxPipe - 1) / kMaxPipe;
}

// The graph of this step of the batch (captured on first use), or null when the step cannot
// be captured (then it runs directly, and so does every later step of this lead).
template <typename R>
BatchGraph* batch_graph(qsa_handle* const* hs, int nh, int nbr, int nbc) {
  qsa_handle* lead = hs[0];
  std::vector<uint64_t> serials(nh);
  std::vector<int64_t> phases(nh);
  for (int i = 0; i < nh; ++i) {
    serials[i] = hs[i]->serial;
    phases[i] = hs[i]->pushes % (int64_t)S<R>(hs[i])->srcs.size();
  }
  for (BatchGraph* g : lead->graphs)
    if (g->nbr == nbr && g->nbc == nbc && g->serials == serials && g->phases == phases) return g;
  if (lead->graphs.size() >= 64) {  // keyed by serials: stale entries only cost memory
    for (BatchGraph* g : lead->graphs) delete g;
    lead->graphs.clear();
  }
  auto* g = new BatchGraph;
  g->serials = serials;
  g->phases = phases;
  g->nbr = nbr;
  g->nbc = nbc;
  const int nl = (nh + kMaxPipe - 1) / kMaxPipe;
  for (int c = 0; c < nl; ++c) {
    void* t = nullptr;
    if (cudaMallocHost(&t, sizeof(PipeTable<R>)) != cudaSuccess) {
      delete g;
      cudaGetLastError();
      return nullptr;
    }
    g->tables.push_back(t);
  }
  // Capture on the lead's own capture stream (the handles' stream may be the legacy default
  // stream, which cannot be captured): the handles issue to it for the capture's duration,
  // and the graph is then launched on their stream.  Each launch uploads its table from its
  // pinned buffer, which the graph reads at every replay.
  if (!lead->cap_stream &&
      cudaStreamCreateWithFlags(&lead->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return nullptr;
  }
  std::vector<PipeTable<R>*> pins(nl);
  for (int c = 0; c < nl; ++c) pins[c] = static_cast<PipeTable<R>*>(g->tables[c]);
  std::vector<cudaStream_t> saved(nh);
  for (int i = 0; i < nh; ++i) {
    saved[i] = hs[i]->stream;
    hs[i]->stream = lead->cap_stream;
  }
  cudaGraph_t graph = nullptr;
  int failed = 0;
  bool ok = cudaStreamBeginCapture(lead->cap_stream, cudaStreamCaptureModeThreadLocal) ==
            cudaSuccess;
  if (ok) {
    ok = issue_batch_step<R>(hs, nh, nbr, nbc, pins.data(), &failed) == QSA_OK;
    g->ev_end = lead->n_timed;
    const cudaError_t e = cudaStreamEndCapture(lead->cap_stream, &graph);
    ok = ok && e == cudaSuccess && graph != nullptr;
  }
  for (int i = 0; i < nh; ++i) hs[i]->stream = saved[i];
  if (ok) ok = cudaGraphInstantiate(&g->exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();  // a capture that failed leaves no error behind for later calls
    for (int i = 0; i < nh; ++i) hs[i]->err.clear();
    delete g;
    return nullptr;
  }
  lead->graphs.push_back(g);
  return g;
}


// n_steps steps of every handle, each launch advancing up to kMaxPipe handles by one step.
// With n_steps >= 2 x (shapes) and no earlier choice, the first steps time each FFT unit
// shape on the real work (every shape computes the same steps) and the rest use the fastest.
// After those, each step runs as a CUDA graph (captured once per distinct step, see
// batch_graph) unless graphs are off for the lead or a capture failed.
template <typename R>
int advance_batch(qsa_handle* const* hs, int nh, int n_steps) {
  qsa_handle* lead = hs[0];
  State<R>* ls = S<R>(lead);
  // a failure in a call made for another handle is reported through the lead
  auto relay = [&](int rc, int i) {
    if (hs[i] != lead) lead->err = "instance " + std::to_string(i) + ": " + hs[i]->err;
    return rc;
  };
  for (int i = 0; i < nh; ++i)
    if (!hs[i]->src_valid)
      if (int rc = deposit_sources<R>(hs[i])) return relay(rc, i);
  const int nl = (nh + kMaxPipe - 1) / kMaxPipe;
  std::vector<PipeTable<R>> tv(nl);  // ~33 KB each: on the heap
  const int nshape = 4;
  const bool tune = ls->tuned_nbr == 0 && n_steps >= 2 * nshape;
  std::vector<float> shape_ms(nshape, 0.f);
  for (int step = 0; step < n_steps; ++step) {
    int nbr = ls->tuned_nbr ? ls->tuned_nbr : kPipeRowBatch;
    int nbc = ls->tuned_nbc ? ls->tuned_nbc : kPipeColBatch;
    const bool timing = tune && step < nshape;
    if (timing) {
      nbr = kTuneShapes[step][0];
      nbc = kTuneShapes[step][1];
      lead->n_timed = 0;
    }
    // graphs once the lazy set-up of the launches (slot table, events) exists
    BatchGraph* g = nullptr;
    if (!timing && lead->batch_graphs && !lead->graphs_failed && ls->ptab && lead->ev[0]) {
      g = batch_graph<R>(hs, nh, nbr, nbc);
      if (!g) lead->graphs_failed = true;
    }
    if (g) {
      qsa_handle* h = lead;  // error reporting of CK
      CK(cudaGraphLaunch(g->exec, lead->stream));
      ++lead->graph_replays;
      // its launch events, re-recorded by this replay, count for qsa_launch_times
      lead->n_timed = std::max(lead->n_timed, g->ev_end);
    } else {
      std::vector<PipeTable<R>*> tp(nl);
      for (int c = 0; c < nl; ++c) tp[c] = &tv[c];
      int failed = 0;
      if (int rc = issue_batch_step<R>(hs, nh, nbr, nbc, tp.data(), &failed))
        return relay(rc, failed);
    }
    finish_batch_step<R>(hs, nh);
    if (timing) {
      qsa_handle* h = lead;  // error reporting of CK
      float tot = 0.f, ms = 0.f;
      for (int i = 0; i < lead->n_timed; ++i) {
        CK(cudaEventSynchronize(lead->ev[2 * i + 1]));
        CK(cudaEventElapsedTime(&ms, lead->ev[2 * i], lead->ev[2 * i + 1]));
        tot += ms;
      }
      shape_ms[step] = tot;
      if (step == nshape - 1) {
        int best = 0;
        for (int k = 1; k < nshape; ++k)
          if (shape_ms[k] < shape_ms[best]) best = k;
        ls->tuned_nbr = kTuneShapes[best][0];
        ls->tuned_nbc = kTuneShapes[best][1];
      }
    }
  }
  return QSA_OK;
}

template <typename R>
int beam_step(qsa_handle* h) {
  State<R>* s = S<R>(h);
  const DevParams& dp = h->dp;
  R* src = ring_src<R>(h, h->pushes + 1);
  int* cmax = ring_cmax<R>(h, h->pushes + 1);
  double* mom = ring_mom<R>(h, h->pushes + 1);
  const R* slab = s->slots[s->last_slot].slab;
  CK(cudaMemsetAsync(src, 0, (size_t)dp.nk * dp.nx * dp.ny * 4 * sizeof(R), h->stream));
  if (int rc = clear_ring<R>(h, h->pushes + 1)) return rc;
  for (size_t si = 0; si < s->beams.size(); ++si) {
    const auto& b = s->beams[si];
    if (b.n == 0) continue;
    const unsigned groups = (unsigned)(s->species[si].nkb * dp.ny);
    beam_kernel<R, true><<<groups, kThreads, beam_smem_bytes<R>(dp.nx), h->stream>>>(
        b, dp, s->species[si], s->bconst[si], slab, src, s->lost,
        Extent{cmax, nullptr, mom + si * (size_t)dp.nxi * 7, nullptr});
    ++h->launches;
    CK(cudaGetLastError());
  }
  ++h->pushes;
  h->src_valid = true;
  return QSA_OK;
}

template <typename R>
int diagnostics(qsa_handle* h, qsa_diag* out) {
  State<R>* s = S<R>(h);
  const int nk = h->dp.nk;
  std::vector<double> d((size_t)D_COUNT * nk);
  int st = 0;
  unsigned long long lost = 0;
  const SweepArgs<R>& a = s->slots[s->last_slot];
  CK(cudaMemcpyAsync(d.data(), a.diag, d.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(&st, a.bar.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&lost, s->lost, sizeof(lost), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  auto row = [&](int r) { return d.data() + (size_t)r * nk; };
  const double npc = (double)h->dp.ppc * h->dp.nx * h->dp.ny;
  for (int j = 0; j < nk; ++j) {
    if (out->energy)
      for (int f = 0; f < 6; ++f) out->energy[(size_t)j * 6 + f] = row(D_E0 + f)[j];
    if (out->psi0) out->psi0[j] = row(D_PSI0)[j];
    if (out->ez0) out->ez0[j] = row(D_EZ0)[j];
    if (out->jz_mean) out->jz_mean[j] = row(D_JZ)[j];
    if (out->kappa2) out->kappa2[j] = row(D_KAPPA)[j] / npc;
    if (out->opp_min) out->opp_min[j] = row(D_OPPMIN)[j];
    if (out->n_floor) out->n_floor[j] = row(D_NFLOOR)[j];
    if (out->invariant) out->invariant[j] = row(D_INV)[j];
    if (out->charge) out->charge[j] = std::fabs(row(D_CHARGE)[j]);
    if (out->pc_residual) {
      const double den = row(D_PCDEN)[j];
      out->pc_residual[j] = den > 0 ? std::sqrt(row(D_PCNUM)[j] / den) : 0.0;
    }
    if (out->pc_iters) out->pc_iters[j] = row(D_NPC)[j];
  }
  // rms fields per slice, and over xi segments: <F^2> = 2 E / (Lx Ly dxi)
  {
    const double ms_norm = 2.0 / (h->dp.Lx * h->dp.Ly * h->dp.dxi);
    const double W = out->seg_width > 0 ? out->seg_width : 2.0;
    const int nseg = std::max(1, (int)std::ceil(h->dp.Lxi / W - 1e-12));
    std::vector<double> acc((size_t)nseg * 6, 0.0), cnt(nseg, 0.0);
    for (int j = 0; j < nk; ++j) {
      const int sgi = std::min(nseg - 1, (int)std::floor(j * h->dp.dxi / W + 1e-12));
      cnt[sgi] += 1.0;
      for (int f = 0; f < 6; ++f) {
        const double ms = row(D_E0 + f)[j] * ms_norm;
        if (out->rms) out->rms[(size_t)j * 6 + f] = std::sqrt(ms);
        acc[(size_t)sgi * 6 + f] += ms;
      }
    }
    if (out->rms_seg)
      for (int sgi = 0; sgi < nseg; ++sgi)
        for (int f = 0; f < 6; ++f)
          out->rms_seg[(size_t)sgi * 6 + f] =
              cnt[sgi] > 0 ? std::sqrt(acc[(size_t)sgi * 6 + f] / cnt[sgi]) : 0.0;
  }
  if (out->mode_amp && h->dp.nmodes > 0) {
    std::vector<R> mo((size_t)nk * h->dp.nmodes * 10);
    CK(cudaMemcpyAsync(mo.data(), a.mode_out, mo.size() * sizeof(R), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (size_t i = 0; i < mo.size(); ++i) out->mode_amp[i] = (double)mo[i];
  }
  if (out->beam_moments && h->prm.n_species > 0) {
    CK(cudaMemcpyAsync(out->beam_moments, ring_mom<R>(h, h->pushes), mom_bytes(h),
                       cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  out->beam_lost = (int64_t)lost;
  out->sweeps = h->sweeps;
  const int rc = status_code(st);
  if (rc < 0) fail(h, rc, status_text(rc));
  return rc;
}

template <typename R>
int copy_field(qsa_handle* h, int field, int j0, int j1, double* out, bool source) {
  State<R>* s = S<R>(h);
  const DevParams& dp = h->dp;
  const int stride = source ? 4 : 8;
  const size_t g = (size_t)dp.nx * dp.ny;
  std::vector<R> tmp((size_t)(j1 - j0) * g * stride);
  const R* base = (source ? ring_src<R>(h, h->pushes) : s->slots[s->last_slot].slab) +
                  (size_t)j0 * g * stride;
  CK(cudaMemcpyAsync(tmp.data(), base, tmp.size() * sizeof(R), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < (size_t)(j1 - j0) * g; ++i) out[i] = (double)tmp[i * stride + field];
  if (source && (field == 0 || field == 1)) {  // add the uniform reference left out of the slab
    const std::vector<double>& ref = field == 0 ? s->bref_s : s->bref_jz;
    for (int j = j0; j < j1; ++j)
      for (size_t i = 0; i < g; ++i) out[(size_t)(j - j0) * g + i] += ref[j];
  }
  return QSA_OK;
}

// Flags (in *bad) a live particle (w != 0) whose xi is outside [0, Lxi), NaN included.
__global__ void check_xi_kernel(const double* __restrict__ xi, const double* __restrict__ w,
                                long long n, double Lxi, int* bad) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n && w[i] != 0.0 && !(xi[i] >= 0.0 && xi[i] < Lxi)) *bad = 1;
}

template <typename R>
int beam_io(qsa_handle* h, int si, bool to_host, int64_t n, const double* const* in,
            double* const* out) {
  State<R>* s = S<R>(h);
  const auto& b = s->beams[si];
  const size_t bytes = (size_t)b.n * sizeof(double);
  std::vector<void*> tmp;
  for (int k = 0; k < 7; ++k) {
    void* p = dalloc(h, bytes);
    if (!p) return fail(h, QSA_ERR_OOM, "beam staging");
    tmp.push_back(p);
  }
  const unsigned blocks = (unsigned)((b.n + kThreads - 1) / kThreads);
  int rc = QSA_OK;
  if (!to_host) {
    for (int k = 0; k < 7; ++k)
      CK(cudaMemcpyAsync(tmp[k], in[k], bytes, cudaMemcpyHostToDevice, h->stream));
    // every live particle's xi must lie in [0, Lxi): checked on the device copy before the
    // beam is touched, so that a rejected call leaves the beam as it was
    int bad = 0;
    CK(cudaMemsetAsync(s->chk, 0, sizeof(int), h->stream));
    check_xi_kernel<<<blocks, kThreads, 0, h->stream>>>((const double*)tmp[2],
                                                        (const double*)tmp[6], b.n,
                                                        h->prm.Lxi, s->chk);
    ++h->launches;
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&bad, s->chk, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (bad) {
      rc = fail(h, QSA_ERR_ARG, "xi of a live particle outside [0, Lxi)");
    } else {
      h->beam_replaced = true;
      h->last_pushes = 0;
      beam_from_host_kernel<R><<<blocks, kThreads, 0, h->stream>>>(
          b, h->dp, s->species[si], (double*)tmp[0], (double*)tmp[1], (double*)tmp[2],
          (double*)tmp[3], (double*)tmp[4], (double*)tmp[5], (double*)tmp[6]);
      ++h->launches;
      CK(cudaGetLastError());
      h->src_valid = false;
    }
  } else {
    beam_to_host_kernel<R><<<blocks, kThreads, 0, h->stream>>>(
        b, h->dp, s->species[si], (double*)tmp[0], (double*)tmp[1], (double*)tmp[2],
        (double*)tmp[3], (double*)tmp[4], (double*)tmp[5], (double*)tmp[6]);
    ++h->launches;
    CK(cudaGetLastError());
    for (int k = 0; k < 7; ++k)
      CK(cudaMemcpyAsync(out[k], tmp[k], bytes, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  // release the staging buffers (the last seven allocations)
  for (int k = 0; k < 7; ++k) {
    auto a = h->allocs.back();
    h->allocs.pop_back();
    h->bytes -= (int64_t)a.second;
    if (h->free_fn) h->free_fn(a.first, a.second, h->ctx, (void*)h->stream);
    else cudaFreeAsync(a.first, h->stream);
  }
  CK(cudaStreamSynchronize(h->stream));
  return rc;
}

template <typename R>
int field_solve(qsa_handle* h, const double* const* in, double kappa2, double* out) {
  State<R>* s = S<R>(h);
  const DevParams& dp = h->dp;
  const size_t g = (size_t)dp.nx * dp.ny;
  SweepArgs<R> a = s->slots[0];
  a.src = nullptr;
  a.bref = nullptr;
  std::vector<R> ov(g * kNF);
  std::vector<double> dg((size_t)D_COUNT * dp.nk, 0.0);
  dg[(size_t)D_KAPPA * dp.nk] = kappa2 * dp.ppc * (double)dp.nx * dp.ny;
  CK(cudaMemcpyAsync(a.diag, dg.data(), dg.size() * sizeof(double), cudaMemcpyHostToDevice,
                     h->stream));
  CK(cudaMemsetAsync(a.part, 0, (size_t)dp.ny * kTileRows * dp.nx * kNF * sizeof(R), h->stream));
  CK(cudaMemsetAsync(a.jprev, 0, 2 * (size_t)dp.nxh * dp.ny * sizeof(C<R>), h->stream));
  CK(cudaMemsetAsync(a.bold, 0, 2 * (size_t)dp.nxh * dp.ny * sizeof(C<R>), h->stream));
  // B solve: trial fields Jx, Jy, Jz, Jx^{+1/2} = D_x dxi, Jy^{+1/2} = D_y dxi (J^{-1/2} = 0),
  // placed field-major in the overflow grid
  for (size_t i = 0; i < g; ++i) {
    ov[0 * g + i] = R(in[1][i]);
    ov[1 * g + i] = R(in[2][i]);
    ov[2 * g + i] = R(in[3][i]);
    ov[3 * g + i] = R(in[4][i] * dp.dxi);
    ov[4 * g + i] = R(in[5][i] * dp.dxi);
  }
  CK(cudaMemcpyAsync(a.ovf, ov.data(), ov.size() * sizeof(R), cudaMemcpyHostToDevice,
                     h->stream));
  // the inputs sit in the overflow grid: every overflow row is read, no outer tile row
  CK(cudaMemsetAsync(a.odirty, 1, (size_t)dp.ny * sizeof(int), h->stream));
  CK(cudaMemsetAsync(a.cflag, 0, (size_t)dp.ny * sizeof(int), h->stream));
  CK(cudaMemsetAsync(a.bar.count, 0, sizeof(unsigned), h->stream));
  int which = 0;
  void* args[] = {&a, &which};
  CK(cudaLaunchCooperativeKernel((void*)solve_kernel<R>, dim3(s->grid), dim3(kThreads), args,
                                 s->smem, h->stream));
  ++h->launches;
  std::vector<R> tmp(g * kFG);
  auto get = [&](const int* comps, double* const* o, int n) -> int {
    CK(cudaMemcpyAsync(tmp.data(), a.fg, g * kFG * sizeof(R), cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int c = 0; c < n; ++c)
      for (size_t i = 0; i < g; ++i) o[c][i] = (double)tmp[i * kFG + comps[c]];
    return QSA_OK;
  };
  int rc;
  {
    const int comps[4] = {FG_EZ, FG_BZ, FG_BX, FG_BY};
    double* const o[4] = {out + 3 * g, out + 4 * g, out + 5 * g, out + 6 * g};
    if ((rc = get(comps, o, 4))) return rc;
  }
  // psi solve: S in field 0 of three
  std::fill(ov.begin(), ov.end(), R(0));
  for (size_t i = 0; i < g; ++i) ov[i] = R(in[0][i]);
  CK(cudaMemcpyAsync(a.ovf, ov.data(), g * 3 * sizeof(R), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(a.odirty, 1, (size_t)dp.ny * sizeof(int), h->stream));
  CK(cudaMemsetAsync(a.part, 0, (size_t)dp.ny * kTileRows * dp.nx * kNF * sizeof(R), h->stream));
  CK(cudaMemsetAsync(a.bar.count, 0, sizeof(unsigned), h->stream));
  which = 1;
  CK(cudaLaunchCooperativeKernel((void*)solve_kernel<R>, dim3(s->grid), dim3(kThreads), args,
                                 s->smem, h->stream));
  ++h->launches;
  {
    const int comps[3] = {FG_PSI, FG_GX, FG_GY};
    double* const o[3] = {out, out + g, out + 2 * g};
    if ((rc = get(comps, o, 3))) return rc;
  }
  int st = 0;
  CK(cudaMemcpyAsync(&st, a.bar.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  // the solve has no slab to check: a non-finite value among its outputs is reported as the
  // sweep reports a non-finite slab value
  for (size_t i = 0; i < 7 * g; ++i)
    if (!std::isfinite(out[i])) {
      st |= ST_NONFINITE;
      break;
    }
  rc = status_code(st);
  return rc < 0 ? fail(h, rc, status_text(rc)) : QSA_OK;
}

// ---- the discrete adjoint (FP64 handles)

// Doubles of one flat copy of every species' beam state (ox, oy, oxi, ux, uy, uz, dw).
size_t beam_doubles(qsa_handle* h) {
  size_t n = 0;
  for (const auto& b : S<double>(h)->beams) n += 7 * (size_t)b.n;
  return n;
}
// Views of species si's arrays inside a flat copy.
BeamArrays<double> beam_view(qsa_handle* h, double* base, int si) {
  State<double>* s = S<double>(h);
  size_t off = 0;
  for (int k = 0; k < si; ++k) off += 7 * (size_t)s->beams[k].n;
  BeamArrays<double> v{};
  const size_t n = (size_t)s->beams[si].n;
  v.n = (long long)n;
  double* q = base + off;
  v.ox = q; v.oy = q + n; v.oxi = q + 2 * n; v.ux = q + 3 * n; v.uy = q + 4 * n;
  v.uz = q + 5 * n; v.dw = q + 6 * n;
  return v;
}
// Copy the handle's beam to a flat copy (to_copy) or back.
int beam_copy(qsa_handle* h, double* flat, bool to_copy) {
  State<double>* s = S<double>(h);
  for (size_t si = 0; si < s->beams.size(); ++si) {
    const BeamArrays<double>& b = s->beams[si];
    const BeamArrays<double> v = beam_view(h, flat, (int)si);
    const size_t by = (size_t)b.n * sizeof(double);
    double* hs[7] = {b.ox, b.oy, b.oxi, b.ux, b.uy, b.uz, b.dw};
    double* cs[7] = {v.ox, v.oy, v.oxi, v.ux, v.uy, v.uz, v.dw};
    for (int k = 0; k < 7; ++k)
      CK(cudaMemcpyAsync(to_copy ? cs[k] : hs[k], to_copy ? hs[k] : cs[k], by,
                         cudaMemcpyDeviceToDevice, h->stream));
  }
  return QSA_OK;
}

void grad_release(qsa_handle* h) {
  if (!h->grad) return;
  for (double* p : h->grad->beam_ckpt) dfree(h, p);
  if (h->grad->beam_end) dfree(h, h->grad->beam_end);
  delete h->grad;
  h->grad = nullptr;
}

int grad_forward(qsa_handle* h, int n_steps, int ckpt, double* loss_out) {
  State<double>* s = S<double>(h);
  const DevParams& dp = h->dp;
  grad_release(h);
  h->grad = new GradRun();
  GradRun& G = *h->grad;
  G.n_steps = n_steps;
  G.ckpt = ckpt;
  const size_t nb = beam_doubles(h);
  auto save = [&](std::vector<double*>& v) -> int {
    double* c = (double*)dalloc(h, nb * sizeof(double));
    if (!c) return fail(h, QSA_ERR_OOM, "beam checkpoint");
    v.push_back(c);
    return beam_copy(h, c, true);
  };
  if (int rc = save(G.beam_ckpt)) return rc;
  for (int n = 0; n < n_steps; ++n) {
    if (int rc = sweep<double>(h)) return rc;
    if (int rc = beam_step<double>(h)) return rc;
    if ((n + 1) % ckpt == 0 && n + 1 < n_steps)
      if (int rc = save(G.beam_ckpt)) return rc;
  }
  if (!(G.beam_end = (double*)dalloc(h, nb * sizeof(double))))
    return fail(h, QSA_ERR_OOM, "beam checkpoint");
  if (int rc = beam_copy(h, G.beam_end, true)) return rc;
  if (int rc = sweep<double>(h)) return rc;
  // the loss of the final sweep, and the status of every sweep of the run
  double* dl = (double*)dalloc(h, sizeof(double));
  if (!dl) return fail(h, QSA_ERR_OOM, "loss");
  CK(cudaMemsetAsync(dl, 0, sizeof(double), h->stream));
  const size_t ncell = (size_t)dp.nk * dp.nx * dp.ny;
  bperp_loss_kernel<<<std::min<size_t>((ncell + 255) / 256, 4096), 256, 0, h->stream>>>(
      s->slots[0].slab, ncell, dp.dx * dp.dy * dp.dxi, 0.0, nullptr, dl);
  ++h->launches;
  CK(cudaGetLastError());
  int st = 0;
  CK(cudaMemcpyAsync(&G.loss, dl, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&st, s->slots[0].bar.status, sizeof(int), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  dfree(h, dl);
  if (st & ST_FLOOR)
    return fail(h, QSA_ERR_STATE, "the psi floor was met: the adjoint takes it as inactive");
  const int rc = status_code(st);
  if (rc < 0) return fail(h, rc, status_text(rc));
  G.pushes = h->pushes;
  G.sweeps = h->sweeps;
  *loss_out = G.loss;
  return QSA_OK;
}

int grad_backward(qsa_handle* h, double dloss, double* dmodes, double* dalpha) {
  State<double>* s = S<double>(h);
  const DevParams& dp = h->dp;
  GradRun& G = *h->grad;
  const int N = G.n_steps, K = G.ckpt, nk = dp.nk, n_pc = dp.n_pc;
  const size_t g = (size_t)dp.nx * dp.ny, np = (size_t)dp.np, spec = (size_t)dp.nxh * dp.ny;
  const size_t nb = beam_doubles(h);
  const int seg = std::min(K, N) + 1;  // sweeps of the longest segment
  std::vector<void*> mine;
  bool oom = false;
  auto A = [&](size_t bytes) -> double* {
    void* p = dalloc(h, bytes);
    if (!p) oom = true;
    else mine.push_back(p);
    return (double*)p;
  };
  auto release = [&]() {
    for (auto it = mine.rbegin(); it != mine.rend(); ++it) dfree(h, *it);
    mine.clear();
  };
  // segment store: tapes, slabs, beam states, per-sweep psi0 and kappa^2
  const size_t tp = (size_t)nk * 5 * np, tf = (size_t)nk * (n_pc + 1) * g * kFG,
               tj = (size_t)nk * 2 * spec;
  std::vector<double*> tpart(seg), tfg(seg), slabs(seg), beams(seg), psi0s(seg), kaps(seg);
  std::vector<C<double>*> tjp(seg);
  for (int i = 0; i < seg; ++i) {
    tpart[i] = A(tp * sizeof(double));
    tfg[i] = A(tf * sizeof(double));
    tjp[i] = (C<double>*)A(tj * sizeof(C<double>));
    slabs[i] = A((size_t)nk * g * 8 * sizeof(double));
    beams[i] = A(nb * sizeof(double));
    psi0s[i] = A((size_t)nk * sizeof(double));
    kaps[i] = A((size_t)nk * sizeof(double));
  }
  // adjoint buffers
  AdjArgs a{};
  a.p = dp;
  a.w = dp.dx * dp.dy / dp.ppc;
  a.idx = 1.0 / dp.dx;
  a.idy = 1.0 / dp.dy;
  a.dv = 1.0 / (dp.dx * dp.dy);
  a.inv_LxLy = 1.0 / (dp.Lx * dp.Ly);
  double* lslab = A((size_t)nk * g * 8 * sizeof(double));
  a.lslab = lslab;
  a.lsrc = A((size_t)nk * g * 4 * sizeof(double));
  const size_t npart_adj = 9 * np, ngrid_adj = 22 * g;
  double* pa = A(npart_adj * sizeof(double));
  double* ga = A(ngrid_adj * sizeof(double));
  a.zs = (C<double>*)A(8 * g * sizeof(C<double>));
  a.zt = (C<double>*)A(8 * g * sizeof(C<double>));
  // beam adjoints (positions, momenta, weight) of every species
  double* lbeam = A(nb * sizeof(double));
  double* gout = A(17 * (size_t)std::max(1, (int)s->species.size()) * sizeof(double));
  if (oom) {
    release();
    return fail(h, QSA_ERR_OOM, "adjoint buffers");
  }
  if (pa) {
    double** pp[9] = {&a.lx, &a.ly, &a.lux, &a.luy, &a.lpp, &a.lopp, &a.loph, &a.lgx, &a.lgy};
    for (int k = 0; k < 9; ++k) *pp[k] = pa + (size_t)k * np;
  }
  {
    double* q = ga;
    for (int b = 0; b < 2; ++b)
      for (int k = 0; k < 3; ++k) { a.lpsi[b][k] = q; q += g; }
    for (int b = 0; b < 2; ++b)
      for (int k = 0; k < 3; ++k) { a.lB[b][k] = q; q += g; }
    for (int b = 0; b < 2; ++b)
      for (int k = 0; k < 2; ++k) { a.ljp[b][k] = q; q += g; }
    a.lS = q; q += g;
    for (int k = 0; k < 5; ++k) { a.lJ[k] = q; q += g; }
  }
  a.twx = s->slots[0].twx;
  a.twy = s->slots[0].twy;
  a.ktab = s->slots[0].ktab;
  a.bar = s->slots[0].bar;
  const size_t asmem = adj_smem_bytes(dp.nx, dp.ny);
  CK(raise_dyn_smem((const void*)adj_sweep_kernel, asmem));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_sweep_kernel, kThreads, asmem));
  if (per_sm < 1) {
    release();
    return fail(h, QSA_ERR_ARG, "adjoint kernel does not fit on an SM");
  }
  const int agrid = per_sm * h->num_sms;
  double* part = A((size_t)agrid * 4 * sizeof(double));
  if (oom) {
    release();
    return fail(h, QSA_ERR_OOM, "adjoint buffers");
  }
  a.part = part;
  // the beam adjoint, as per-species views of lbeam
  auto ladj = [&](int si) {
    const BeamArrays<double> v = beam_view(h, lbeam, si);
    return BeamAdj{v.ox, v.oy, v.oxi, v.ux, v.uy, v.uz, v.dw};
  };
  CK(cudaMemsetAsync(lbeam, 0, nb * sizeof(double), h->stream));
  CK(cudaMemsetAsync(gout, 0, 17 * std::max<size_t>(1, s->species.size()) * sizeof(double),
                     h->stream));
  const double npc = (double)dp.ppc * dp.nx * dp.ny;
  std::vector<double> diag((size_t)D_COUNT * nk), kv(nk);
  const int nseg = (N + K) / K;  // segments start at 0, K, 2K, ... <= N
  for (int m = nseg - 1; m >= 0; --m) {
    const int n0 = m * K, n1 = std::min(n0 + K, N + 1);
    // recompute the segment from its checkpoint, recording every sweep
    // the state a segment starts from: a checkpoint, or the end state for a segment that
    // holds only the final sweep
    double* ck = (n0 == N) ? G.beam_end : G.beam_ckpt[m];
    if (int rc = beam_copy(h, ck, false)) { release(); return rc; }
    h->src_valid = false;
    for (int n = n0; n < n1; ++n) {
      const int i = n - n0;
      SweepArgs<double>& sa = s->slots[0];
      sa.tape = Tape<double>{tpart[i], tfg[i], tjp[i]};
      int rc = sweep<double>(h);
      sa.tape = Tape<double>{nullptr, nullptr, nullptr};
      if (rc) { release(); return rc; }
      CK(cudaMemcpyAsync(slabs[i], sa.slab, (size_t)nk * g * 8 * sizeof(double),
                         cudaMemcpyDeviceToDevice, h->stream));
      if ((rc = beam_copy(h, beams[i], true))) { release(); return rc; }
      CK(cudaMemcpyAsync(diag.data(), sa.diag, diag.size() * sizeof(double),
                         cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int j = 0; j < nk; ++j) kv[j] = diag[(size_t)D_KAPPA * nk + j] / npc;
      CK(cudaMemcpyAsync(psi0s[i], diag.data() + (size_t)D_PSI0 * nk, nk * sizeof(double),
                         cudaMemcpyHostToDevice, h->stream));
      CK(cudaMemcpyAsync(kaps[i], kv.data(), nk * sizeof(double), cudaMemcpyHostToDevice,
                         h->stream));
      CK(cudaStreamSynchronize(h->stream));
      if (n < N)
        if ((rc = beam_step<double>(h))) { release(); return rc; }
    }
    // backwards through the segment
    for (int n = n1 - 1; n >= n0; --n) {
      const int i = n - n0;
      if (n == N) {
        const size_t ncell = (size_t)nk * g;
        bperp_loss_kernel<<<std::min<size_t>((ncell + 255) / 256, 4096), 256, 0, h->stream>>>(
            slabs[i], ncell, dp.dx * dp.dy * dp.dxi, dloss, lslab, nullptr);
        ++h->launches;
      } else {
        // push n: beam state n through slab n gives beam state n + 1
        CK(cudaMemsetAsync(lslab, 0, (size_t)nk * g * 8 * sizeof(double), h->stream));
        for (size_t si = 0; si < s->beams.size(); ++si) {
          const BeamArrays<double> b = beam_view(h, beams[i], (int)si);
          if (b.n == 0) continue;
          beam_push_adj_kernel<<<(unsigned)((b.n + kThreads - 1) / kThreads), kThreads, 0,
                                 h->stream>>>(b, dp, s->species[si], slabs[i], lslab,
                                              ladj((int)si));
          ++h->launches;
        }
      }
      CK(cudaGetLastError());
      // the sweep of step n
      CK(cudaMemsetAsync(a.lsrc, 0, (size_t)nk * g * 4 * sizeof(double), h->stream));
      CK(cudaMemsetAsync(pa, 0, npart_adj * sizeof(double), h->stream));
      CK(cudaMemsetAsync(ga, 0, ngrid_adj * sizeof(double), h->stream));
      CK(cudaMemsetAsync(a.bar.count, 0, sizeof(unsigned), h->stream));
      a.tape = Tape<double>{tpart[i], tfg[i], tjp[i]};
      a.psi0 = psi0s[i];
      a.kappa2 = kaps[i];
      void* args[] = {&a};
      CK(cudaLaunchCooperativeKernel((void*)adj_sweep_kernel, dim3(agrid), dim3(kThreads), args,
                                     asmem, h->stream));
      ++h->launches;
      // the beam sources of step n, deposited from beam state n
      for (size_t si = 0; si < s->beams.size(); ++si) {
        const BeamArrays<double> b = beam_view(h, beams[i], (int)si);
        if (b.n == 0) continue;
        beam_src_adj_kernel<<<(unsigned)((b.n + kThreads - 1) / kThreads), kThreads, 0,
                              h->stream>>>(b, dp, s->species[si], a.lsrc, ladj((int)si));
        ++h->launches;
      }
      CK(cudaGetLastError());
    }
  }
  // weights -> mode amplitudes and alpha, per species
  for (size_t si = 0; si < s->beams.size(); ++si) {
    const BeamArrays<double> b0 = beam_view(h, G.beam_ckpt[0], (int)si);
    if (b0.n == 0) continue;
    weight_grad_kernel<<<(unsigned)((b0.n + kThreads - 1) / kThreads), kThreads, 0,
                         h->stream>>>(b0.dw, b0.n, dp, s->species[si], s->modes,
                                      ladj((int)si).lw, gout + 17 * si);
    ++h->launches;
  }
  CK(cudaGetLastError());
  std::vector<double> go(17 * std::max<size_t>(1, s->species.size()));
  int st = 0;
  CK(cudaMemcpyAsync(go.data(), gout, go.size() * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaMemcpyAsync(&st, a.bar.status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  // leave the handle as the forward run left it
  if (int rc = beam_copy(h, G.beam_end, false)) { release(); return rc; }
  CK(cudaStreamSynchronize(h->stream));
  release();
  h->pushes = G.pushes;
  h->sweeps = G.sweeps;
  h->src_valid = false;
  const int nm = s->modes.n;
  if (dmodes)
    for (int k = 0; k < nm; ++k) {
      dmodes[k] = 0.0;
      for (size_t si = 0; si < s->species.size(); ++si) dmodes[k] += go[17 * si + k];
    }
  if (dalpha)
    for (size_t si = 0; si < s->species.size(); ++si) dalpha[si] = go[17 * si + nm];
  const int rc = status_code(st);
  return rc < 0 ? fail(h, rc, status_text(rc)) : QSA_OK;
}

int validate(const qsa_params* p, std::string& why) {
  auto bad = [&](const std::string& m) { why = m; return QSA_ERR_ARG; };
  if (!p) return bad("params is NULL");
  if (!size_ok(p->nx) || !size_ok(p->ny)) return bad("nx, ny must be 1 or 2^a 3^b <= 512");
  if (p->nxi < 1) return bad("nxi must be >= 1");
  if (!(p->Lx > 0 && p->Ly > 0 && p->Lxi > 0 && p->dt > 0)) return bad("box and dt must be > 0");
  if (p->ppc_plasma_x < 1 || p->ppc_plasma_y < 1 || p->ppc_plasma_x * p->ppc_plasma_y > 64)
    return bad("plasma ppc must be in 1..64");
  if (p->n_species < 0 || p->n_species > QSA_MAX_SPECIES) return bad("n_species out of range");
  if (p->n_modes < 0 || p->n_modes > QSA_MAX_MODES) return bad("n_modes out of range");
  if (p->precision != QSA_FP64 && p->precision != QSA_MIXED) return bad("unknown precision");
  if (p->n_pc_iter < 1 || p->n_pc_iter > 64) return bad("n_pc_iter must be in 1..64");
  if (!(p->pc_tol >= 0.0 && p->pc_tol <= 1e100)) return bad("pc_tol must be finite and >= 0");
  if (!(p->rehome_frac >= 0.0 && p->rehome_frac <= 1.0)) return bad("rehome_frac must be in [0, 1]");
  if (!(p->psi_floor > 0 && p->psi_floor < 1)) return bad("psi_floor must be in (0, 1)");
  if (p->spin_limit < 0) return bad("spin_limit must be >= 0");
  if (p->pipeline_depth < 0 || p->pipeline_depth > kMaxPipe)
    return bad("pipeline_depth must be in 0..16");
  if (p->n_diag_modes < 0 || p->n_diag_modes > QSA_MAX_MODES)
    return bad("n_diag_modes must be in 0..16");
  for (int m = 0; m < p->n_diag_modes; ++m) {
    const qsa_kvec k = p->diag_modes[m];
    if (k.mx == 0 && k.my == 0) return bad("diag mode k = 0 (psi0, E_z0 are separate outputs)");
    if (2 * std::abs(k.mx) > p->nx || 2 * std::abs(k.my) > p->ny)
      return bad("diag mode beyond the Nyquist index");
  }
  const double dxi = p->Lxi / p->nxi;
  for (int s = 0; s < p->n_species; ++s) {
    const qsa_species& q = p->species[s];
    if (!(q.M > 0) || !(q.gamma_b >= 1) || !(q.alpha > 0)) return bad("species M/gamma/alpha");
    if (q.ppc_x < 1 || q.ppc_y < 1 || q.ppc_xi < 1) return bad("species ppc must be >= 1");
    const double back = q.xi_back < 0 ? p->Lxi : q.xi_back;
    if (q.xi_front < 0 || back > p->Lxi * (1 + 1e-12) || back <= q.xi_front)
      return bad("species xi extent must satisfy 0 <= front < back <= Lxi");
    if (std::fabs(q.xi_front / dxi - std::lround(q.xi_front / dxi)) > 1e-9 ||
        std::fabs(back / dxi - std::lround(back / dxi)) > 1e-9)
      return bad("species xi extent must be whole slices");
    if (!(q.gamma_spread_rel >= 0 && q.gamma_spread_rel < 0.2)) return bad("gamma spread");
  }
  return QSA_OK;
}

}  // namespace

namespace {
// An NVTX range around each call of the C ABI, so that a timeline tool shows which call a
// launch or a copy belongs to (NVTX is header-only: without a tool attached it costs a
// few nanoseconds per call).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace

extern "C" {

int qsa_init(const qsa_params* params, void* stream, qsa_alloc_fn alloc, qsa_free_fn free_fn,
             void* alloc_ctx, qsa_handle** out) {
  NvtxRange nvtx_range("qsa_init");
  if (!out) return fail(nullptr, QSA_ERR_ARG, "out is NULL");
  *out = nullptr;
  std::string why;
  if (validate(params, why) != QSA_OK) return fail(nullptr, QSA_ERR_ARG, why);
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(nullptr, QSA_ERR_ARG, "alloc and free must both be given or both be NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, QSA_ERR_CUDA, cudaGetErrorString(e));
  qsa_handle* h = new qsa_handle();
  static std::atomic<uint64_t> next_serial{1};
  h->serial = next_serial++;
  h->prm = *params;
  h->stream = (cudaStream_t)stream;
  h->alloc = alloc;
  h->free_fn = free_fn;
  h->ctx = alloc_ctx;
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  DevParams& dp = h->dp;
  dp.nx = params->nx;
  dp.ny = params->ny;
  dp.nxi = params->nxi;
  dp.nk = params->nxi + 1;
  dp.nxh = params->nx / 2 + 1;
  dp.ppx = params->ppc_plasma_x;
  dp.ppy = params->ppc_plasma_y;
  dp.ppc = dp.ppx * dp.ppy;
  dp.np = dp.ppc * dp.nx * dp.ny;
  dp.n_pc = params->n_pc_iter;
  dp.pc_tol2 = params->pc_tol * params->pc_tol;
  dp.nsmem_rows = kTileRows;
  dp.Lx = params->Lx;
  dp.Ly = params->Ly;
  dp.Lxi = params->Lxi;
  dp.dx = params->Lx / params->nx;
  dp.dy = params->Ly / params->ny;
  dp.dxi = params->Lxi / params->nxi;
  dp.dt = params->dt;
  dp.psi_floor = params->psi_floor;
  dp.spin_limit = params->spin_limit;
  dp.px = make_plan(dp.nx);
  dp.py = make_plan(dp.ny);
  dp.fd_nx = make_fastdiv(dp.nx);
  dp.fd_ny = make_fastdiv(dp.ny);
  dp.fd_nxh = make_fastdiv(dp.nxh);
  // diagnosed modes on the half spectrum: k itself when mx >= 0, else its conjugate -k
  dp.nmodes = params->n_diag_modes;
  for (int m = 0; m < dp.nmodes; ++m) {
    const qsa_kvec k = params->diag_modes[m];
    const int sg = k.mx < 0 ? -1 : 1;
    dp.mkx[m] = sg * k.mx;
    dp.mky[m] = ((sg * k.my) % dp.ny + dp.ny) % dp.ny;
    dp.mconj[m] = k.mx < 0 ? 1 : 0;
  }
  h->fp64 = params->precision == QSA_FP64;
  const size_t smem = h->fp64 ? sweep_smem<double>(dp) : sweep_smem<float>(dp);
  int max_smem = 0;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  int rc;
  if ((int)smem > max_smem) {
    rc = fail(h, QSA_ERR_ARG, "grid too large for shared memory");
  } else {
    rc = h->fp64 ? setup<double>(h) : setup<float>(h);
  }
  if (rc != QSA_OK) {
    g_init_error = h->err;
    qsa_destroy(h);
    return rc;
  }
  *out = h;
  return QSA_OK;
}

int qsa_set_beam(qsa_handle* h, int s, int64_t n, const double* x, const double* y,
                 const double* xi, const double* ux, const double* uy, const double* uz,
                 const double* w) {
  NvtxRange nvtx_range("qsa_set_beam");
  if (!h) return QSA_ERR_ARG;
  if (s < 0 || s >= h->prm.n_species) return fail(h, QSA_ERR_ARG, "species index");
  const int64_t want = h->fp64 ? S<double>(h)->beams[s].n : S<float>(h)->beams[s].n;
  if (n != want) return fail(h, QSA_ERR_ARG, "n must equal the species' lattice count");
  if (!x || !y || !xi || !ux || !uy || !uz || !w) return fail(h, QSA_ERR_ARG, "NULL array");
  const double* in[7] = {x, y, xi, ux, uy, uz, w};
  return h->fp64 ? beam_io<double>(h, s, false, n, in, nullptr)
                 : beam_io<float>(h, s, false, n, in, nullptr);
}

int qsa_get_beam(qsa_handle* h, int s, int64_t cap, double* x, double* y, double* xi,
                 double* ux, double* uy, double* uz, double* w, int64_t* n_out) {
  NvtxRange nvtx_range("qsa_get_beam");
  if (!h) return QSA_ERR_ARG;
  if (s < 0 || s >= h->prm.n_species) return fail(h, QSA_ERR_ARG, "species index");
  const int64_t n = h->fp64 ? S<double>(h)->beams[s].n : S<float>(h)->beams[s].n;
  if (cap < n) return fail(h, QSA_ERR_ARG, "capacity smaller than the species count");
  if (!x || !y || !xi || !ux || !uy || !uz || !w) return fail(h, QSA_ERR_ARG, "NULL array");
  double* out[7] = {x, y, xi, ux, uy, uz, w};
  const int rc = h->fp64 ? beam_io<double>(h, s, true, n, nullptr, out)
                         : beam_io<float>(h, s, true, n, nullptr, out);
  if (n_out) *n_out = rc == QSA_OK ? n : 0;
  return rc;
}

int qsa_plasma_sweep(qsa_handle* h) {
  NvtxRange nvtx_range("qsa_plasma_sweep");
  if (!h) return QSA_ERR_ARG;
  return h->fp64 ? sweep<double>(h) : sweep<float>(h);
}

int qsa_beam_step(qsa_handle* h) {
  NvtxRange nvtx_range("qsa_beam_step");
  if (!h) return QSA_ERR_ARG;
  if (h->sweeps == 0) return fail(h, QSA_ERR_STATE, "beam step before any sweep");
  return h->fp64 ? beam_step<double>(h) : beam_step<float>(h);
}

int qsa_advance(qsa_handle* h, int32_t n_steps) {
  NvtxRange nvtx_range("qsa_advance");
  if (!h) return QSA_ERR_ARG;
  if (n_steps < 0) return fail(h, QSA_ERR_ARG, "n_steps must be >= 0");
  if (h->prm.pipeline_depth > 1) {
    h->n_timed = 0;
    return h->fp64 ? advance_pipelined<double>(h, n_steps) : advance_pipelined<float>(h, n_steps);
  }
  for (int32_t i = 0; i < n_steps; ++i) {
    int rc = h->fp64 ? sweep<double>(h) : sweep<float>(h);
    if (rc) return rc;
    rc = h->fp64 ? beam_step<double>(h) : beam_step<float>(h);
    if (rc) return rc;
  }
  return QSA_OK;
}

int qsa_advance_batch(qsa_handle* const* handles, int32_t n_handles, int32_t n_steps) {
  NvtxRange nvtx_range("qsa_advance_batch");
  if (!handles || n_handles < 1) return fail(nullptr, QSA_ERR_ARG, "no handles");
  qsa_handle* lead = handles[0];
  if (!lead) return fail(nullptr, QSA_ERR_ARG, "NULL handle");
  if (n_steps < 0) return fail(lead, QSA_ERR_ARG, "n_steps must be >= 0");
  for (int i = 0; i < n_handles; ++i) {
    const qsa_handle* h = handles[i];
    if (!h) return fail(lead, QSA_ERR_ARG, "NULL handle");
    if (h->fp64 != lead->fp64) return fail(lead, QSA_ERR_ARG, "handles differ in precision");
    if (h->stream != lead->stream) return fail(lead, QSA_ERR_ARG, "handles differ in stream");
    if (h->dp.n_pc != lead->dp.n_pc) return fail(lead, QSA_ERR_ARG, "handles differ in n_pc_iter");
    if (h->dp.pc_tol2 != lead->dp.pc_tol2)
      return fail(lead, QSA_ERR_ARG, "handles differ in pc_tol");
    for (int k = 0; k < i; ++k)
      if (handles[k] == h) return fail(lead, QSA_ERR_ARG, "a handle appears twice");
  }
  lead->n_timed = 0;
  return lead->fp64 ? advance_batch<double>(handles, n_handles, n_steps)
                    : advance_batch<float>(handles, n_handles, n_steps);
}

int qsa_batch_graphs(qsa_handle* lead, int32_t enable, int64_t* replays) {
  NvtxRange nvtx_range("qsa_batch_graphs");
  if (!lead) return fail(nullptr, QSA_ERR_ARG, "NULL handle");
  if (enable > 0) {
    lead->batch_graphs = true;
    lead->graphs_failed = false;
  } else if (enable == 0) {
    lead->batch_graphs = false;
  }
  if (replays) *replays = lead->batch_graphs && !lead->graphs_failed ? lead->graph_replays
                                                                      : -1 - lead->graph_replays;
  return QSA_OK;
}

int qsa_diagnostics(qsa_handle* h, qsa_diag* out) {
  NvtxRange nvtx_range("qsa_diagnostics");
  if (!h || !out) return QSA_ERR_ARG;
  return h->fp64 ? diagnostics<double>(h, out) : diagnostics<float>(h, out);
}

int qsa_copy_field(qsa_handle* h, int field, int j0, int j1, double* host_out) {
  NvtxRange nvtx_range("qsa_copy_field");
  if (!h || !host_out) return QSA_ERR_ARG;
  if (field < 0 || field > 5 || j0 < 0 || j1 > h->dp.nk || j0 >= j1)
    return fail(h, QSA_ERR_ARG, "field or slice range");
  return h->fp64 ? copy_field<double>(h, field, j0, j1, host_out, false)
                 : copy_field<float>(h, field, j0, j1, host_out, false);
}

int qsa_copy_source(qsa_handle* h, int q, int j0, int j1, double* host_out) {
  NvtxRange nvtx_range("qsa_copy_source");
  if (!h || !host_out) return QSA_ERR_ARG;
  if (q < 0 || q > 3 || j0 < 0 || j1 > h->dp.nk || j0 >= j1)
    return fail(h, QSA_ERR_ARG, "source or node range");
  if (!h->src_valid) {
    const int rc = h->fp64 ? deposit_sources<double>(h) : deposit_sources<float>(h);
    if (rc) return rc;
  }
  return h->fp64 ? copy_field<double>(h, q, j0, j1, host_out, true)
                 : copy_field<float>(h, q, j0, j1, host_out, true);
}

int qsa_field_solve(qsa_handle* h, const double* S_, const double* Jx, const double* Jy,
                    const double* Jz, const double* Dx, const double* Dy, double kappa2,
                    double* out) {
  NvtxRange nvtx_range("qsa_field_solve");
  if (!h || !S_ || !Jx || !Jy || !Jz || !Dx || !Dy || !out) return QSA_ERR_ARG;
  if (!(kappa2 >= 0)) return fail(h, QSA_ERR_ARG, "kappa2 must be >= 0");
  const double* in[6] = {S_, Jx, Jy, Jz, Dx, Dy};
  return h->fp64 ? field_solve<double>(h, in, kappa2, out) : field_solve<float>(h, in, kappa2, out);
}

int qsa_rehome(qsa_handle* h) {
  NvtxRange nvtx_range("qsa_rehome");
  if (!h) return QSA_ERR_ARG;
  return h->fp64 ? rehome<double>(h) : rehome<float>(h);
}

int64_t qsa_rehome_count(const qsa_handle* h) { return h ? h->rehomes : 0; }

int qsa_grad_forward(qsa_handle* h, int32_t n_steps, int32_t step_ckpt, double* loss_out) {
  NvtxRange nvtx_range("qsa_grad_forward");
  if (!h || !loss_out) return QSA_ERR_ARG;
  if (!h->fp64) return fail(h, QSA_ERR_ARG, "the adjoint needs an FP64 handle");
  if (n_steps < 0 || step_ckpt < 1) return fail(h, QSA_ERR_ARG, "n_steps >= 0, step_ckpt >= 1");
  if (h->dp.pc_tol2 > 0.0)
    return fail(h, QSA_ERR_ARG, "the adjoint needs a fixed predictor-corrector count (pc_tol 0)");
  if (h->pushes != 0 || h->sweeps != 0)
    return fail(h, QSA_ERR_STATE, "the run must start from the beam qsa_init built");
  if (h->beam_replaced)
    return fail(h, QSA_ERR_STATE, "the beam was replaced: the weights no longer follow the "
                                  "mode amplitudes and alpha");
  const int rc = grad_forward(h, n_steps, step_ckpt, loss_out);
  if (rc) grad_release(h);
  return rc;
}

int qsa_grad_backward(qsa_handle* h, double dloss, double* dl_dmodes, double* dl_dalpha) {
  NvtxRange nvtx_range("qsa_grad_backward");
  if (!h) return QSA_ERR_ARG;
  if (!h->grad) return fail(h, QSA_ERR_STATE, "no run recorded by qsa_grad_forward");
  const int rc = grad_backward(h, dloss, dl_dmodes, dl_dalpha);
  grad_release(h);
  return rc;
}

int qsa_phase_times(qsa_handle* h, int64_t* out, int cap) {
  if (!h || !out) return QSA_ERR_ARG;
  const int n = kTimedSlices * kTimedPhases * 2;
  if (cap < n) return fail(h, QSA_ERR_ARG, "capacity below 512");
  unsigned long long* dev =
      h->fp64 ? S<double>(h)->slots[0].ptimes : S<float>(h)->slots[0].ptimes;
  CK(cudaMemcpyAsync(out, dev, n * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return QSA_OK;
}

int qsa_launch_times(qsa_handle* h, float* ms, int cap, int* n_out) {
  if (!h || !ms || !n_out) return QSA_ERR_ARG;
  *n_out = 0;
  const int n = h->n_timed < cap ? h->n_timed : cap;
  for (int i = 0; i < n; ++i) {
    CK(cudaEventSynchronize(h->ev[2 * i + 1]));
    CK(cudaEventElapsedTime(ms + i, h->ev[2 * i], h->ev[2 * i + 1]));
  }
  *n_out = n;
  return QSA_OK;
}

int64_t qsa_launch_count(const qsa_handle* h) { return h ? h->launches : 0; }

int64_t qsa_device_bytes(const qsa_handle* h) { return h ? h->bytes : 0; }

const char* qsa_last_error(const qsa_handle* h) {
  return h ? h->err.c_str() : g_init_error.c_str();
}

int qsa_bounds_check(int64_t* first_line, int64_t* count) {
  if (first_line) *first_line = 0;
  if (count) *count = 0;
#ifdef QSA_DEBUG_BOUNDS
  // this file's counters (the persistent kernels) and those of the allocation-free solve's
  // file; the Eq. 5 solver's file holds no index checks
  unsigned long long f = 0, c = 0, fs = 0, cs = 0;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpyFromSymbol(&f, qsa::g_bounds_first, sizeof(f)) != cudaSuccess ||
      cudaMemcpyFromSymbol(&c, qsa::g_bounds_count, sizeof(c)) != cudaSuccess ||
      qsa::static_bounds_counts(&fs, &cs) != QSA_OK)
    return QSA_ERR_CUDA;
  if (first_line) *first_line = (int64_t)(f ? f : fs);
  if (count) *count = (int64_t)(c + cs);
  return 1;
#else
  return 0;
#endif
}

void qsa_destroy(qsa_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  delete h->grad;  // its buffers go with every other allocation below
  h->grad = nullptr;
  dfree_all(h);
  cudaStreamSynchronize(h->stream);
  if (h->st) {
    if (h->fp64) delete S<double>(h);
    else delete S<float>(h);
  }
  for (int i = 0; i < 2 * qsa_handle::kLaunchEvents; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  for (BatchGraph* g : h->graphs) delete g;
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

}  // extern "C"
