/*
 * qsa.h -- C ABI of the B300 quasistatic PIC (QS-PIC) hot path.
 *
 * The method: arxiv 2607.24214, "Modeling ultrarelativistic streaming plasma instabilities
 * under the quasistatic approximation".  Its section "Quasistatic model" fixes the physical
 * setting (cold plasma electrons, immobile ions, beam species of charge Z_s, mass M_s, density
 * ratio alpha_s = n_bs/n_p and Lorentz factor gamma_b; comoving variables (xi, tau) =
 * (ct - x, t)); its QuaSSis paragraph fixes the code family (QS-PIC, transversely periodic
 * boundaries, random macroparticle weights).  The paper prints no discrete algorithm; the
 * discrete scheme implemented here (and, independently, by the FP64 oracle under oracle/) is:
 *   - per beam step, a plasma sweep over xi slices j = 0..nxi: the plasma electrons start at
 *     rest on a quiet lattice at xi = 0 and are pushed slice by slice; at each slice the
 *     transverse fields psi, E_z, B_z, B_x, B_y are solved spectrally on the periodic grid, B_perp
 *     by a predictor-corrector of n_pc_iter solves; the k = 0 mode is integrated in FP64;
 *   - then a beam push by dt (relativistic Boris) through the stored slice fields.
 * Normalised units throughout: time 1/omega_p, length c/omega_p, momentum m_e c, density n_p,
 * fields m_e c omega_p/e.  z is the propagation axis; the paper's x is z here, its y is (x, y).
 *
 * Conventions of every entry point
 *   - All calls return a qsa_status (0 = QSA_OK, < 0 error, > 0 warning) unless stated.
 *   - Host arrays passed in are copied before the call returns; output buffers are the
 *     caller's.  The library owns all device memory; it allocates it through the caller's
 *     allocator callbacks when given (else cudaMallocAsync on the handle's stream).
 *   - Work is enqueued on the handle's stream (the cudaStream_t passed to qsa_init, may be 0).
 *     Calls that return host data synchronise that stream.
 *   - Device-side failures (a grid barrier that timed out, non-finite values) are latched in a
 *     device status word and returned by the next synchronising call.
 *   - One handle per stream; a handle is not thread-safe.
 *   - On error, qsa_last_error(h) gives a one-line description.
 */
#ifndef QSA_H
#define QSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QSA_MAX_SPECIES 4
#define QSA_MAX_MODES 16
#define QSA_MAX_N 512 /* largest transverse grid side: sizes are 1 or 2^a 3^b <= 512 */

typedef enum {
  QSA_OK = 0,
  QSA_ERR_ARG = -1,       /* invalid argument or parameter */
  QSA_ERR_CUDA = -2,      /* a CUDA runtime call failed */
  QSA_ERR_OOM = -3,       /* an allocation failed */
  QSA_ERR_TIMEOUT = -4,   /* a device-side wait exceeded spin_limit iterations */
  QSA_ERR_NONFINITE = -5, /* non-finite field or particle value detected */
  QSA_ERR_STATE = -6,     /* call out of order (e.g. beam step before any sweep) */
  QSA_WARN_PSI_FLOOR = 1  /* 1 + psi fell below psi_floor for some plasma particle */
} qsa_status;

typedef enum { QSA_FP64 = 0, QSA_MIXED = 1 } qsa_precision;

/* One beam species (section "Quasistatic model": Z_s, M_s, alpha_s, gamma_b). */
typedef struct {
  double Z, M, alpha, gamma_b;
  double gamma_spread_rel; /* std of gamma/gamma_b (Gaussian) */
  double uperp_spread;     /* std of u_x, u_y (Gaussian, m_e c) */
  double noise_rel;        /* std of the relative weight perturbation ("random weights") */
  int32_t ppc_x, ppc_y, ppc_xi;
  int32_t seeded;          /* 1: multiply this species' weights by the mode list */
  double xi_front, xi_back;/* beam occupies [xi_front, xi_back); xi_back < 0 means Lxi */
} qsa_species;

/* A transverse wave vector k = (2 pi mx / Lx, 2 pi my / Ly). */
typedef struct {
  int32_t mx, my;
} qsa_kvec;

/* Seeded transverse density mode: weight factor 1 + amplitude cos(k.x + phase). */
typedef struct {
  int32_t mx, my;          /* k = (2 pi mx / Lx, 2 pi my / Ly) */
  double amplitude, phase;
} qsa_mode;

typedef struct {
  int32_t nx, ny, nxi;     /* transverse cells (1 or 2^a 3^b <= 512), xi slices */
  int32_t ppc_plasma_x, ppc_plasma_y;
  int32_t n_species, n_modes;
  int32_t precision;       /* qsa_precision */
  int32_t n_pc_iter;       /* predictor-corrector field solves per slice (>= 1) */
  int32_t pipeline_depth;  /* beam steps one qsa_advance launch keeps in flight (0, 1: none;
                              2..16: pipelined, see qsa_advance) */
  double Lx, Ly, Lxi;      /* periodic box (Lx, Ly) and window length, c/omega_p */
  double dt;               /* beam time step, 1/omega_p */
  double psi_floor;        /* lower bound applied to 1 + psi of plasma particles */
  uint64_t seed;           /* Philox key of the beam initial conditions */
  int64_t spin_limit;      /* iteration limit of every device-side wait */
  qsa_species species[QSA_MAX_SPECIES];
  qsa_mode modes[QSA_MAX_MODES];
  int32_t n_diag_modes;    /* transverse modes whose amplitude every sweep records (0..16) */
  int32_t _pad;
  qsa_kvec diag_modes[QSA_MAX_MODES]; /* k != 0, |mx| <= nx/2, |my| <= ny/2 */
  double pc_tol;           /* 0: exactly n_pc_iter field solves per slice.  > 0: the B_perp
                              predictor-corrector (part of the QS-PIC scheme, whose discrete
                              steps the paper does not print) iterated to a tolerance: stop
                              after the first solve whose relative change
                              ||B_perp(n) - B_perp(n-1)|| / ||B_perp(n)|| (2-norms over the
                              grid) is below pc_tol, after n_pc_iter solves at most; the
                              count per slice is reported in qsa_diag.pc_iters */
  double rehome_frac;      /* qsa_advance with pipeline_depth >= 2: before a persistent launch,
                              when more than this fraction of the beam sat outside its storage
                              slots' cells after the previous launch's pushes, re-home the beam
                              (move each particle into a slot of the cell it occupies, within
                              its xi layer; each keeps its identity for qsa_get_beam).  The
                              sources and fields are unchanged up to the order of the sums.
                              0: never.  Storage only, not part of the method. */
} qsa_params;

/* Allocator callbacks: alloc returns a device pointer (NULL on failure) of at least `bytes`
 * bytes, aligned to 256 B, usable on `stream`; free releases it. */
typedef void* (*qsa_alloc_fn)(size_t bytes, void* ctx, void* stream);
typedef void (*qsa_free_fn)(void* ptr, size_t bytes, void* ctx, void* stream);

typedef struct qsa_handle qsa_handle;

/* Per-slice diagnostics of the last sweep; every non-NULL pointer is a caller array of
 * nxi + 1 entries unless stated (energy: 6 * (nxi + 1), slice-major).  Any pointer may be
 * NULL.  The field amplitudes and the beam moments are those of the paper's growth and
 * saturation figures: rms fields over the transverse plane and over xi segments of width
 * 2 k_p^-1 (Fig. 2), Fourier amplitudes of single modes (the growth rates of Eq. 5), and the
 * beam's rms momentum spread per xi position (Fig. 3f). */
typedef struct {
  double* energy;       /* 1/2 sum F^2 dx dy dxi of E_x, E_y, E_z, B_x, B_y, B_z */
  double* psi0;         /* k = 0 mode of psi */
  double* ez0;          /* k = 0 mode of E_z */
  double* jz_mean;      /* <J_z> total (plasma + beam) */
  double* kappa2;       /* Helmholtz shift of the B_perp solves, <w/(1+psi)>/(Lx Ly) */
  double* opp_min;      /* min over plasma particles of 1 + psi (before the floor) */
  double* n_floor;      /* plasma particles with 1 + psi < psi_floor */
  double* invariant;    /* max |gamma - u_z - (1+psi)|/(1+psi) */
  double* charge;       /* |sum_cells (rho - J_z)_plasma dx dy + Lx Ly| */
  double* pc_residual;  /* ||B_perp(n) - B_perp(n-1)|| / ||B_perp(n)|| of the last solve */
  int64_t beam_lost;    /* out: beam particles that left the window (all species) */
  int64_t sweeps;       /* out: sweeps done by this handle */
  double* rms;          /* [nxi+1][6]: sqrt(<F^2>) over the transverse plane of E_x, E_y, E_z,
                           B_x, B_y, B_z (from the energies) */
  double seg_width;     /* in: xi width of the rms_seg segments; <= 0 means 2 k_p^-1 */
  double* rms_seg;      /* [ceil(Lxi / seg_width)][6]: sqrt of <F^2> averaged over the
                           transverse plane and the slices j dxi of segment s, i.e.
                           s seg_width <= j dxi < (s+1) seg_width (slice nxi joins the last) */
  double* mode_amp;     /* [nxi+1][n_diag_modes][5][2]: Fourier coefficient F(k)/(nx ny)
                           (re, im; F(x) = sum_k F(k) e^{i k.x} / (nx ny), forward transform
                           with e^{-i k.x}) of psi, E_z, B_x, B_y, B_z at each slice */
  double* beam_moments; /* [n_species][nxi][7]: over the live particles whose xi lies in cell
                           c, sums of w/wbar, (w/wbar) u_x, (w/wbar) u_y, (w/wbar) du_z,
                           (w/wbar) u_x^2, (w/wbar) u_y^2, (w/wbar) du_z^2, with
                           du_z = u_z - sqrt(gamma_b^2 - 1) and wbar the species' nominal
                           weight; of the current beam (after the last push) */
  double* pc_iters;     /* field solves of the predictor-corrector at each slice (n_pc_iter
                           unless pc_tol > 0) */
} qsa_diag;

/* Create a handle for the setting of section "Quasistatic model" (plasma electrons, immobile
 * ions, beam species Z_s, M_s, alpha_s, gamma_b) with the random macroparticle weights of the
 * QuaSSis paragraph (section "Extending the QSA to extreme blazar jet regimes").
 * Validates params, allocates device state, builds every beam species on
 * the device from `seed` (quiet lattice, Philox-4x32-10 random weights and momenta; the same
 * construction as paper_2607_24214_b300/inputs.py).  `stream` is a cudaStream_t or NULL.
 * alloc/free may be NULL (then cudaMallocAsync / cudaFreeAsync).  Errors: QSA_ERR_ARG for an
 * invalid parameter, QSA_ERR_OOM, QSA_ERR_CUDA; *out is NULL on error. */
int qsa_init(const qsa_params* params, void* stream, qsa_alloc_fn alloc, qsa_free_fn free_fn,
             void* alloc_ctx, qsa_handle** out);

/* The beam macroparticles of the QS-PIC (QuaSSis paragraph): their state is all a resumed run
 * needs, since the plasma is rebuilt at xi = 0 every sweep (section "Quasistatic model").
 * Replace species `s` with host fp64 arrays of n particles in the canonical id order of the
 * lattice (id = ((k_xi*ny + iy)*nx + ix)*ppc + (s_xi*ppc_y + s_y)*ppc_x + s_x); n must equal
 * the species' lattice count.  x, y in [0, L); xi in [0, Lxi); w = 0 marks a lost particle.
 * Copies and converts to the device layout; marks the beam sources stale.  QSA_ERR_ARG when
 * a live particle's xi is outside [0, Lxi) (checked on the device copy before the beam is
 * touched: the beam stays as it was).  Synchronises. */
int qsa_set_beam(qsa_handle* h, int s, int64_t n, const double* x, const double* y,
                 const double* xi, const double* ux, const double* uy, const double* uz,
                 const double* w);

/* The beam state of the QS-PIC (QuaSSis paragraph), read back.
 * Copy species `s` back to host fp64 arrays (canonical id order, positions wrapped into
 * [0, L)); cap = capacity of each array; *n_out = particles written.  Synchronises. */
int qsa_get_beam(qsa_handle* h, int s, int64_t cap, double* x, double* y, double* xi,
                 double* ux, double* uy, double* uz, double* w, int64_t* n_out);

/* The quasistatic plasma response (section "Quasistatic model": at fixed tau the fields
 * depend on xi = ct - x; the nonlinear counterparts of Eqs. 1-2 and of the B_perp equations).
 * One plasma sweep at the current beam state: deposits the beam sources if stale, then runs
 * the slice loop j = 0..nxi in one persistent launch and fills the field slab and the
 * per-slice diagnostics.  Asynchronous. */
int qsa_plasma_sweep(qsa_handle* h);

/* The slow evolution of the beam in tau (section "Quasistatic model"; the nonlinear
 * counterpart of Eq. 3).
 * Push every live beam particle by dt through the current field slab (trilinear gather,
 * relativistic Boris), drop particles with xi >= Lxi, and deposit the beam sources of the
 * next sweep.  QSA_ERR_STATE before the first sweep.  Asynchronous. */
int qsa_beam_step(qsa_handle* h);

/* The QS-PIC time loop (QuaSSis paragraph): alternating plasma sweeps and beam pushes.
 * n_steps beam steps, each a plasma sweep followed by a beam push: the same result as
 * n_steps x (qsa_plasma_sweep; qsa_beam_step), up to the summation order of the deposits.
 * With pipeline_depth S >= 2 the steps run in persistent launches of up to S steps each, as a
 * wavefront in xi: the sweep of a step trails the previous step by a few slices, since its
 * slice j needs only the beam sources of nodes <= j + 1, which are final once the previous
 * step has pushed every particle that can land there (beam particles only move backwards in
 * the window; the gates follow the particles' actual xi extent per layer, so the schedule is
 * exact for any drift).  The work of the steps in flight is spread over every SM in each
 * phase.  Memory: S sweep slots (each one field slab of (nxi+1) nx ny 8 values) and S + 1
 * source buffers.  Afterwards the slab and the diagnostics are those of the last sweep and
 * the sources those of the next.  n_steps = 0 is a no-op.  Asynchronous. */
int qsa_advance(qsa_handle* h, int32_t n_steps);

/* Parameter scans over alpha_b and gamma_b, like the scan after Fig. 2 (section "Analytical
 * solutions") that finds the 0.4 N_e filamentation extent independent of both.
 * n_steps beam steps (sweep + push) of each of n_handles independent instances, which may
 * differ in grid size, beam, box and every other parameter except precision, n_pc_iter,
 * pc_tol and stream (the same for all; a handle may appear once).  Each step of up to 16 instances runs
 * in one persistent launch whose phases cover the work of all of them (parameter scans over
 * alpha and gamma_b).  The same result per instance as n_steps x (qsa_plasma_sweep;
 * qsa_beam_step) on it, up to the summation order of the deposits.  The FFT work units (rows
 * and half-spectrum columns per unit) are chosen by timing: with n_steps >= 8 and no earlier
 * choice for handles[0], the first 4 steps run one candidate shape each (all compute the same
 * steps) and the remaining steps use the fastest; the choice is kept in handles[0].  Device-
 * side failures (timeouts) of these launches are latched in handles[0].  Uses handles[0]'s
 * launch timing (qsa_launch_times).  Asynchronous, except during the timing steps. */
int qsa_advance_batch(qsa_handle* const* handles, int32_t n_handles, int32_t n_steps);

/* CUDA graphs of the batched steps (the paper has no counterpart).
 * qsa_advance_batch led by `lead` runs each step after the autotuner's timing steps as a
 * CUDA graph: the step's stream work (slot preparation, the table uploads from pinned host
 * copies, the persistent launches, the diagnostic reductions) is captured once per distinct
 * step (the same handles, FFT unit shape and ring phase of each handle's sources) and
 * replayed; a step whose capture fails runs directly, and so do the later ones.  The
 * results are those of the direct launches.  enable: 1 on (the default; also retries after
 * a failed capture), 0 off, < 0 unchanged.  replays (optional): the number of steps run as
 * graphs so far, or -1 - that number when graphs are off or a capture failed.  With graphs,
 * qsa_launch_times reports the launches of the captured steps' latest replays (and of the
 * call's direct steps). */
int qsa_batch_graphs(qsa_handle* lead, int32_t enable, int64_t* replays);

/* Tracing (the paper has no counterpart).
 * Device time, in ms, of each persistent launch of the last pipelined qsa_advance or
 * qsa_advance_batch call led by h (CUDA events recorded around the launches on the handle's
 * stream; up to 64 launches): writes min(cap, launches) values to ms and their number to
 * *n_out.  0 values when there was none.  Synchronises with those events. */
int qsa_launch_times(qsa_handle* h, float* ms, int cap, int* n_out);

/* Copy the per-slice diagnostics of the last sweep into `out`; synchronises and returns the
 * latched device status (QSA_ERR_TIMEOUT, QSA_WARN_PSI_FLOOR, ...). */
int qsa_diagnostics(qsa_handle* h, qsa_diag* out);

/* The slice fields of section "Quasistatic model" (F_perp = E_y - c B_z of Fig. 1d is
 * E_y + B_x here, in the 3D labels of this library).
 * Copy field `field` (0..5 = E_x - B_y, E_y + B_x, E_z, B_x, B_y, B_z) of slices j0..j1-1
 * of the slab into host_out[(j - j0) * ny * nx + iy * nx + ix] (fp64).  Synchronises. */
int qsa_copy_field(qsa_handle* h, int field, int j0, int j1, double* host_out);

/* The beam charge and current that drive the plasma (rho_b of Eq. 1 and its currents).
 * Copy beam source `q` (0..3 = S_b = Z n (1 - v_z), J_zb, J_xb, J_yb) of nodes j0..j1-1 into
 * host_out like qsa_copy_field.  Deposits the sources first if they are stale. */
int qsa_copy_source(qsa_handle* h, int q, int j0, int j1, double* host_out);

/* The transverse field equations of a slice (Eq. 2's operator for psi and its B_perp and
 * E_z, B_z analogues, section "Quasistatic model").
 * Standalone transverse solve on the handle's grid, through the same device phases (row
 * FFT, column FFT + k-space solve, inverse FFTs) as the sweep.  Inputs are host fp64 [ny][nx]
 * arrays; the k = 0 mode is dropped:
 *   psi = S/k^2, d_x psi, d_y psi;  E_z = -(i k.J)/k^2;  B_z = (i k_x J_y - i k_y J_x)/k^2;
 *   (k^2 + kappa2) B_x = i k_y J_z + D_y,  (k^2 + kappa2) B_y = -i k_x J_z - D_x.
 * out: 7 host arrays back to back, [7][ny][nx]: psi, d_x psi, d_y psi, E_z, B_z, B_x, B_y.
 * Uses the handle's sweep buffers (do not overlap with a sweep); synchronises.  Returns
 * QSA_ERR_NONFINITE if an output is not finite. */
int qsa_field_solve(qsa_handle* h, const double* S, const double* Jx, const double* Jy,
                    const double* Jz, const double* Dx, const double* Dy, double kappa2,
                    double* out);

/* ---------------------------------------------------------------------------------------
 * Linear spatiotemporal theory (Eq. 5), marched on the GPU for a batch of transverse modes:
 * the procedure behind the growth curves of the paper's Fig. 1e.  For each mode m, Eq. 5 with
 * growth rate Gamma_m (Gamma^2 = sum_s omega_bs^2 k^2/(k^2 + 1)) reads
 *   (d_xi^2 + 1) d_tau^2 psi = Gamma_m^2 psi,
 * with zero data ahead of the beam front (xi < 0).  So d_tau^2 psi(xi) =
 * Gamma^2 int_0^xi sin(xi - xi') psi(xi') dxi', evaluated with the trapezoid rule on the grid
 * xi_i = i dxi, i = 0..n_xi-1, and the state (psi, d_tau psi) advances by classical RK4 in tau
 * with n_tau steps of tau_end / n_tau.  FP64 throughout.
 * Arguments: gamma[n_modes]; psi0, dpsi0: psi and d_tau psi at tau = 0, [n_modes][n_xi];
 * psi_out: [n_out][n_modes][n_xi], psi at tau = tau_end (o + 1) / n_out, o = 0..n_out-1
 * (n_out must divide n_tau).  All host arrays (copied; device memory comes from
 * cudaMallocAsync on `stream` and is released before the call returns).  Synchronises.
 * Errors: QSA_ERR_ARG (n_modes < 1, n_xi outside 2..QSA_EQ5_MAX_XI, dxi <= 0, tau_end < 0,
 * n_tau < 1, n_out not dividing n_tau, Gamma < 0, NULL array), QSA_ERR_CUDA; the message is
 * in qsa_last_error(NULL). */
#define QSA_EQ5_MAX_XI 2048
int qsa_eq5_march(int32_t n_modes, int32_t n_xi, double dxi, const double* gamma,
                  const double* psi0, const double* dpsi0, double tau_end, int32_t n_tau,
                  int32_t n_out, double* psi_out, void* stream);

/* ---------------------------------------------------------------------------------------
 * Transverse field solve that allocates nothing.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc (or any allocating routine) when they
 * need a solve, for instance a code whose own memory manager has already reserved the GPU's
 * memory in a fixed pool, or a process running under a hard device-memory budget, where a new
 * allocation would fail or fragment that pool.  Such callers still own their inputs and
 * outputs; only the solve's scratch memory comes from the library.
 *
 * It computes exactly what qsa_field_solve computes (same device kernels), for one grid:
 *   psi = S/k^2, d_x psi, d_y psi;  E_z = -(i k.J)/k^2;  B_z = (i k_x J_y - i k_y J_x)/k^2;
 *   (k^2 + kappa2) B_x = i k_y J_z + D_y,  (k^2 + kappa2) B_y = -i k_x J_z - D_x  (k = 0 dropped).
 * Arguments: nx, ny in {1, 2^a 3^b} and <= QSA_STATIC_MAX_N; periodic box Lx, Ly > 0;
 * kappa2 >= 0; precision QSA_FP64 (arrays of double) or QSA_MIXED (arrays of float); S, Jx,
 * Jy, Jz, Dx, Dy: DEVICE pointers to [ny][nx] arrays; out: DEVICE pointer to [7][ny][nx]
 * (psi, d_x psi, d_y psi, E_z, B_z, B_x, B_y); stream: cudaStream_t of the current device, or
 * NULL.  The call enqueues its work on the stream and returns after synchronising it.
 * Memory: the scratch lives in one file-scope device array of QSA_STATIC_SCRATCH_BYTES that
 * every GPU loading this library holds until the process exits.  The first call on a device
 * takes that array's device address (cudaGetSymbolAddress, with that device current); make
 * that first call before any stream capture.  The call itself calls no cudaMalloc, cudaFree or
 * other allocating routine.  Every call shares the one array and leaves its contents behind
 * (the call clears what must start at zero), so calls that overlap on the GPU - from two
 * streams or two host threads - race and must be serialised by the caller.
 * Errors: QSA_ERR_ARG for a size above QSA_STATIC_MAX_N, an invalid size or argument, or a
 * grid whose scratch would not fit, or a stream of another device (qsa_last_error(NULL) says
 * which); QSA_ERR_CUDA if a CUDA call fails (the failing call and CUDA's text are in
 * qsa_last_error(NULL)); QSA_ERR_TIMEOUT if a device-side wait gave up; QSA_ERR_NONFINITE if an
 * output is not finite (a non-finite input, for instance), as qsa_field_solve reports it. */
#define QSA_STATIC_MAX_N 128
#define QSA_STATIC_SCRATCH_BYTES (6u * 1024u * 1024u + 512u * 1024u)
int qsa_field_solve_static(int32_t nx, int32_t ny, double Lx, double Ly, double kappa2,
                           int32_t precision, const void* S, const void* Jx, const void* Jy,
                           const void* Jz, const void* Dx, const void* Dy, void* out,
                           void* stream);

/* Storage only (the paper has no counterpart): re-home the beam now, moving every particle
 * into a storage slot of the cell it occupies within its xi layer (the ones of a crowded
 * cell fill free slots of other cells, in row-major order), each keeping its identity for
 * qsa_get_beam.  Sources and fields are unchanged up to the order of the sums.  qsa_advance
 * does it by itself when rehome_frac says so.  Uses about 1 GB of staging memory, allocated
 * on first use.  Asynchronous.  qsa_rehome_count: re-homings done by the handle. */
int qsa_rehome(qsa_handle* h);
int64_t qsa_rehome_count(const qsa_handle* h);

/* ---------------------------------------------------------------------------------------
 * Gradients of a run with respect to the seeded mode amplitudes and the beam density ratio
 * (a discrete adjoint of the QS-PIC step).  The paper's linear theory (Eqs. 3-5) makes the
 * growth of every transverse mode depend on alpha and on the seed the beam carries; these
 * calls give d(loss)/d(amplitude of each qsa_mode) and d(loss)/d(alpha of each species) for
 *   loss = 1/2 sum over the slices and cells of the final sweep of (B_x^2 + B_y^2) dx dy dxi,
 * the transverse magnetic (filamentation) energy of the paper's Fig. 2 and Fig. 3d, after
 * n_steps beam steps.  Both enter the run only through the initial macroparticle weights
 * w = wbar (1 + noise) (1 + sum_m a_m cos(k_m . x0 + phi_m)) (wbar proportional to alpha).
 *
 * qsa_grad_forward runs n_steps x (qsa_plasma_sweep; qsa_beam_step) and the final sweep from
 * the beam qsa_init built (the handle must be fresh: no sweep, push or qsa_set_beam before),
 * keeps the beam state every step_ckpt steps (beam-step checkpoints), and writes the loss.
 * qsa_grad_backward then recomputes each segment of step_ckpt steps from its checkpoint,
 * recording every sweep slice by slice (particle state, fields of every field solve), and
 * runs the adjoint backwards: sweep (slices in reverse), beam-source deposit, beam push.  It
 * writes dloss * d(loss)/d(a_m) to dl_dmodes[n_modes] and dloss * d(loss)/d(alpha_s) to
 * dl_dalpha[n_species] (either may be NULL), and leaves the handle as qsa_grad_forward left
 * it.  The adjoint is exact for the discrete scheme (no approximation beyond rounding) when
 * no plasma particle meets the psi floor; qsa_grad_forward returns QSA_ERR_STATE when one
 * does.  Memory: step_ckpt + 1 beam copies and one segment's records (about
 * (step_ckpt + 1) (7 np + 8 (n_pc_iter + 1) nx ny) (nxi + 1) doubles), allocated through
 * the handle's allocator during qsa_grad_backward and released before it returns.
 * Errors: QSA_ERR_ARG (not an FP64 handle, pc_tol > 0, n_steps < 0, step_ckpt < 1),
 * QSA_ERR_STATE (handle not fresh, beam replaced, psi floor met, no recorded run),
 * QSA_ERR_OOM, QSA_ERR_CUDA, and the device status of the sweeps.  Synchronise. */
int qsa_grad_forward(qsa_handle* h, int32_t n_steps, int32_t step_ckpt, double* loss_out);
int qsa_grad_backward(qsa_handle* h, double dloss, double* dl_dmodes, double* dl_dalpha);

/* Tracing (the paper has no counterpart).
 * Phase timing of the last sweep: out[(j * 32 + ph) * 2 + 0] is the device
 * globaltimer (ns) when the last block arrived at the barrier closing phase ph of slice j,
 * out[... + 1] when block 0 left it, for slices j < 8 and phases ph < 32 (trial iteration it,
 * step k in {deposit, row FFT, column FFT + solve, inverse row FFT}: ph = 4 it + k; commit:
 * ph = 4 n_pc_iter + k).  Zero where not recorded.  cap >= 512.  Synchronises. */
int qsa_phase_times(qsa_handle* h, int64_t* out, int cap);

/* Kernel launches made by this handle since qsa_init (launch accounting; the paper has no
 * counterpart). */
int64_t qsa_launch_count(const qsa_handle* h);

/* Device bytes held by the handle (bookkeeping; the paper has no counterpart). */
int64_t qsa_device_bytes(const qsa_handle* h);

/* One-line text of the last error of h (or of the last failed qsa_init, or of the last failed
 * call without a handle, when h is NULL).  The paper has no counterpart. */
const char* qsa_last_error(const qsa_handle* h);

/* Release the handle and all its device memory (waits for its stream).  The paper has no
 * counterpart. */
void qsa_destroy(qsa_handle* h);

/* Bounds checks of the debug build (built with -DQSA_DEBUG_BOUNDS as libqsa_bounds.so; the
 * paper has no counterpart): the index checks at the particle, tile, slab and field-grid
 * accesses of the sweep, push and pipelined kernels and of qsa_field_solve_static record the
 * source line of the first failure and the number of failures on the current device, and
 * skip the access (the counts of both source files are added; the Eq. 5 solver has no
 * index checks).  Writes
 * them to *first_line and *count (each may be NULL) and returns 1 in that build, 0 (with
 * zeros) in the release build, QSA_ERR_CUDA if the counters cannot be read.  Synchronises
 * the device. */
int qsa_bounds_check(int64_t* first_line, int64_t* count);

#ifdef __cplusplus
}
#endif
#endif /* QSA_H */
