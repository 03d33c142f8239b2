/*
 * rmgtd -- real-time TDDFT density-matrix propagation on one GB300 GPU (C ABI).
 *
 * Method: Jakowski et al., "Simulation of 24,000 Electrons Dynamics: Real-Time TDDFT with
 * the Real-Space Multigrids (RMG)", arXiv:2410.09189.  The library implements the time
 * loop of Algorithm 1 (Section 3.1) in a fixed active space of N = N_occ + N_virt
 * orthonormal Kohn-Sham orbitals Phi on a uniform 3-D grid:
 *   - first-order Magnus operator Omega = -i dt (H_0 + H_1)/2 (Eq. 15),
 *   - exp(Omega) applied to the density matrix P by the commutator expansion
 *     dP_k = (Omega dP_{k-1} + dP_{k-1} Omega^dagger)/k until max|dP_k| <= dP_thrs
 *     (Eqs. 19, 33; real/imaginary split of Eq. 35),
 *   - Hamiltonian self-consistency: H_1 <- DFT(rho(P_1)) until max|H_new - H_1| <= H_thrs,
 *     seeded by H_1 = 2 H_0 - H_-1 (Algorithm 1's extrapolation),
 *   - DFT(rho) = density rho(r) = sum_ij Re(P)_ij phi_i phi_j, multigrid Poisson solve for
 *     V_H, LDA exchange-correlation, H = H_core + h^3 Phi^T diag(V_H + V_xc) Phi,
 *   - dipole d_q = Tr(Re(P) M_q), M_q = h^3 Phi^T q Phi (Algorithm 1's dipole),
 *   - delta kick P <- exp(-i kappa M_q) P exp(i kappa M_q) (Eq. 34 with a delta envelope).
 *
 * Conventions (atomic units):
 *   - Grid: point i of an axis with n points sits at (i - (n-1)/2) h (box centre = origin).
 *     A grid function is an array [nz][ny][nx] (x fastest); Ng = nx*ny*nz.
 *   - Orbital blocks are orbital-major: column j of the Ng x N block is contiguous,
 *     element (g, j) at offset j*Ng + g ("Ng x N column-major").
 *   - N x N matrices are row-major doubles.
 *   - Inner products carry the grid quadrature h^3 (Eq. 4), so Phi is orthonormal when
 *     h^3 Phi^T Phi = I.
 *
 * Ownership: every pointer passed to rmgtd_create is read during the call only (inputs
 * are copied).  The context owns all device memory it allocates; host output buffers
 * belong to the caller.  Device pointers passed to rmgtd_apply_h / rmgtd_hartree /
 * rmgtd_xc belong to the caller and must stay valid until the work on the context's
 * stream has finished.
 *
 * Errors: every call returns an rmgtd_status and never aborts; rmgtd_last_error() gives a
 * message.  A failed rmgtd_step leaves the last completed step's state in place.
 *
 * Streams: all work is ordered on the context's stream (rmgtd_options.stream, NULL = the
 * legacy default stream).  Calls that return host data synchronise that stream.
 */
#ifndef RMGTD_H
#define RMGTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rmgtd_ctx rmgtd_ctx;

typedef enum {
  RMGTD_OK = 0,
  RMGTD_EINVAL = -1,         /* bad argument or size */
  RMGTD_ENOMEM = -2,         /* device allocation failed */
  RMGTD_ECUDA = -3,          /* a CUDA runtime call failed */
  RMGTD_ENOTCONVERGED = -4,  /* SCF pass cap or commutator term cap reached */
  RMGTD_EDIVERGED = -5,      /* non-finite value in the series or the SCF error */
  RMGTD_ETIMEOUT = -6,       /* a device-side wait gave up after its iteration limit */
  RMGTD_ESTATE = -7          /* call not valid in the context's current state */
} rmgtd_status;

/* Arithmetic of the propagation path. */
typedef enum {
  RMGTD_PREC_FP64 = 0,   /* every step in float64 */
  RMGTD_PREC_MIXED = 1   /* float32 orbitals and grid contractions, float64 subspace algebra */
} rmgtd_precision;

/* Element type of an orbital block passed to rmgtd_apply_h. */
typedef enum {
  RMGTD_F64 = 0,   /* double */
  RMGTD_F32 = 1,   /* float */
  RMGTD_C128 = 2,  /* complex double, interleaved (re, im) */
  RMGTD_C64 = 3    /* complex float, interleaved (re, im) */
} rmgtd_dtype;

/* Device allocator hook: return `bytes` of device memory usable on `stream` (NULL on
 * failure).  Lets a host framework (e.g. PyTorch's caching allocator) own the memory. */
typedef void* (*rmgtd_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*rmgtd_free_fn)(void* ptr, void* user);

/* The system: grid, pseudo-atoms, active space and starting orbitals (all host memory). */
typedef struct {
  int nx, ny, nz;          /* grid points per axis (each >= 8) */
  double h;                /* grid spacing (bohr) */
  int natoms;
  const double* pos;       /* [natoms][3] positions, origin = box centre */
  const double* Z;         /* [natoms] local-well charges: V_a = -Z erf(r/rc)/r */
  const double* rc_loc;    /* [natoms] erf radii */
  int nproj;               /* Kleinman-Bylander projectors (may be 0) */
  const int* proj_atom;    /* [nproj] owning atom */
  const int* proj_l;       /* [nproj] 0 = s: exp(-r^2/rc^2); 1 = p: (q-R_q) exp(-r^2/rc^2) */
  const int* proj_m;       /* [nproj] p component 0/1/2 = x/y/z (ignored for s) */
  const double* proj_rc;   /* [nproj] Gaussian radii; the projector is cut at r > 5 rc */
  const double* E_kb;      /* [nproj] KB energies (hartree) */
  int nocc, nvirt;         /* active space N = nocc + nvirt */
  const double* f;         /* [N] occupations (NULL: 2 for the first nocc, 0 after) */
  const double* phi0;      /* [N][Ng] starting orbitals (orbital-major), required */
  double v_ext_omega;      /* > 0 adds the harmonic well 0.5 w^2 r^2 (test mode) */
  int hartree_xc;          /* 1: V_eff includes V_H + V_xc; 0: independent electrons */
  const double* rho_core;  /* [Ng] frozen core density (may be NULL): added to rho in the
                              exchange-correlation only (V_xc and eps_xc of rho + rho_core,
                              E_xc = h^3 sum (rho + rho_core) eps_xc), not in the Hartree
                              potential, the dipole or Tr P */
} rmgtd_system;

typedef struct {
  double dt;               /* time step (a.u.) of Algorithm 1 */
  double H_thrs;           /* SCF threshold on max|H_new - H_1| (Algorithm 1) */
  double dP_thrs;          /* commutator-series threshold on max|dP_k| (Algorithm 1) */
  int max_scf;             /* SCF pass cap per step (exceeded -> RMGTD_ENOTCONVERGED) */
  int max_terms;           /* commutator-term cap per expansion */
  int precision;           /* rmgtd_precision */
  int nrep;                /* independent replicas sharing Phi (e.g. 3 kick directions) */
  int orthonormalize;      /* 1: Cholesky-orthonormalise phi0 in float64 on the device */
  double poisson_tol;      /* relative residual of the Hartree solve */
  int poisson_max_iter;    /* PCG iteration cap per Hartree solve */
  int use_graph;           /* 1: run each time step as one captured CUDA graph */
  void* stream;            /* cudaStream_t for all work (NULL = default stream) */
  rmgtd_alloc_fn alloc;    /* NULL: cudaMalloc */
  rmgtd_free_fn free;      /* NULL: cudaFree */
  void* alloc_user;
  int subspace_scf;        /* > 0: up to this many SCF iterations inside the orbital block
                              before t = 0 (P_0 = aufbau projector of H[rho(P_0)], N <= 1024);
                              0: P_0 = diag(f) (the orbitals are taken as the ground state) */
  double subspace_mix;     /* linear mixing of P in those iterations (default 0.3) */
  double subspace_tol;     /* stop when max|P_new - P| <= subspace_tol (default 1e-10) */
  double mixed_poisson_tol;  /* mixed path: relative residual of the float32 Hartree correction
                                solve (0 = default 3e-6; values below 1e-8 are raised to 1e-8) */
  int magnus_order;        /* 1 (or 0): Omega = Omega_1 = -i dt (H_0 + H_1)/2 (Eq. 15);
                              2: plus Omega_2 = (dt^2/12)[H_0, H_1] (Section 2.2, H linear over
                              the step; each H with the external field's value at its end) */
  int nonorthogonal;       /* 1: propagate in the basis phi0 as given (Section 2.2, the series
                              with S^-1 Hbar; Appendix A.2): S = h^3 Phi^T Phi, Omega =
                              -i dt S^-1 (Hbar + V), kicks with S^-1 M_q, start P_0 =
                              L^-T diag(f) L^-1 (S = L L^T), electron count Tr(Re P S).
                              Requires orthonormalize = 0, subspace_scf = 0, magnus_order 1. */
  int grid_basis;          /* 1: propagate the occupied orbitals on the grid, the complete-
                              grid-basis limit of Algorithm 1 (Section 2.2: the scheme holds in
                              any basis).  Per step V_1 = 2 V_0 - V_-1; per SCF pass the series
                              psi^(k) = (-i dt/k) Hbar psi^(k-1), Hbar = T + V_ion + V_NL +
                              (V_0 + V_1)/2 + Ebar.q, stopped at max|psi^(k)| <= dP_thrs; then
                              V_new of rho = sum f |psi|^2 and H_err = max|V_new - V_1| (the grid
                              basis's H_new - H_1 is diagonal); after the loop a float64
                              Cholesky re-orthonormalisation.  The kick is the phase
                              e^{-i kappa q}.  phi0 holds the occupied orbitals: nvirt = 0,
                              magnus_order 1, nonorthogonal 0, subspace_scf 0.  Precision FP64:
                              every step in float64; MIXED: the series terms in float32 (the
                              orbitals, their sum, the fields and the re-orthonormalisation
                              stay float64).
                              rmgtd_kick / set_field / step / dipole / energy / density act on
                              the orbitals (stats: passes, terms of the orbital series,
                              H_err = max|V_new - V_1|); the matrix, save / load, batch,
                              autotune and network calls return RMGTD_ESTATE. */
  int ground_state_scf;    /* > 0: before the set-up, up to this many SCF iterations of the
                              Kohn-Sham ground state on the GPU (Algorithm 1's ground state)
                              from the orthonormalised phi0: Chebyshev-filtered subspace
                              iteration on N + max(4, N/8) orbitals (degree 12 per iteration,
                              Rayleigh-Ritz), Pulay-mixed density (history 6, mixing 0.4); phi0
                              is replaced by the N lowest Kohn-Sham orbitals (ascending energies).  Requires
                              orthonormalize = 1, nonorthogonal = 0, N + buffer <= 1024.
                              RMGTD_ENOTCONVERGED if the cap is reached. */
  double ground_state_tol; /* stop when max|rho_out - rho_in| and the largest Ritz residual
                              max|H phi_n - eps_n phi_n| (n < N) are below it (0: 1e-8) */
  int seed_order;          /* seed of each step's SCF loop: 1 (or 0) the linear extrapolation
                              H_1 = 2 H_0 - H_-1 (Algorithm 1's extrapolation); 2 the quadratic
                              H_1 = 3 H_0 - 3 H_-1 + H_-2 (fewer passes when H varies smoothly;
                              the loop's H_thrs test still decides convergence).  H_-2 starts as
                              H_0, and after rmgtd_load or setting H_-1 it restarts from H_-1.
                              With grid_basis the same seeds act on the potential V. */
  int sm_budget;           /* > 0: every kernel grid of the context, the persistent Hartree and
                              commutator kernels included, is sized to this many SMs instead of
                              the device's; contexts whose budgets sum to at most the SM count
                              then run concurrently inside one rmgtd_batch graph (0: all SMs) */
} rmgtd_options;

/* Per-step, per-replica statistics written by rmgtd_step. */
typedef struct {
  int passes;        /* DFT evaluations (SCF passes) in this step */
  int terms_max;     /* largest number of commutator terms in one expansion */
  int terms_sum;     /* commutator terms summed over the passes */
  int status;        /* rmgtd_status of this replica's step */
  double H_err;      /* final max|H_new - H_1| */
} rmgtd_stats;

/* Matrices readable / writable with rmgtd_get_matrix / rmgtd_set_matrix (N x N doubles). */
typedef enum {
  RMGTD_MAT_P_RE = 0,   /* Re P of the current state (symmetric) */
  RMGTD_MAT_P_IM = 1,   /* Im P of the current state (antisymmetric) */
  RMGTD_MAT_H0 = 2,     /* H at the current time */
  RMGTD_MAT_HM1 = 3,    /* H one step earlier */
  RMGTD_MAT_HCORE = 4,  /* h^3 Phi^T (T + V_loc + V_ext + V_NL) Phi (shared, read-only) */
  RMGTD_MAT_MX = 5,     /* dipole matrices h^3 Phi^T q Phi (shared, read-only) */
  RMGTD_MAT_MY = 6,
  RMGTD_MAT_MZ = 7,
  RMGTD_MAT_S = 8       /* overlap h^3 Phi^T Phi after set-up (shared, read-only) */
} rmgtd_matrix;

/* Fill `opt` with defaults: dt 0.05, H_thrs 1e-7, dP_thrs 1e-10, max_scf 50,
 * max_terms 200, FP64, nrep 1, orthonormalize 1, magnus_order 1, nonorthogonal 0,
 * poisson_tol 1e-12, 200 PCG iterations,
 * use_graph 1 (each time step is one CUDA graph with device-side while loops for the SCF
 * passes and the Hartree iterations), default stream, cudaMalloc. */
void rmgtd_default_options(rmgtd_options* opt);

/* Set up a context (Algorithm 1's set-up given the orbitals): copy Phi, build V_loc and
 * the KB projectors on the device, orthonormalise Phi (optional), form H_core, M_q and the
 * ground-state H_0 = H[rho(P_0)] with P_0 = diag(f) for every replica, H_-1 = H_0.
 * Errors: RMGTD_EINVAL (sizes, NULL required pointers, nrep < 1), RMGTD_ENOMEM,
 * RMGTD_ECUDA.  On failure *out is NULL. */
int rmgtd_create(const rmgtd_system* sys, const rmgtd_options* opt, rmgtd_ctx** out);

/* Free every device buffer of the context (NULL is ignored). */
void rmgtd_destroy(rmgtd_ctx* ctx);

/* hx = H x for `ncols` orbitals on the grid (Eq. 1): -1/2 Lap_12 x + V x + KB part, with
 * Dirichlet-zero ghosts.  V = V_loc + V_ext, plus V_H + V_xc of replica `rep` when rep >= 0
 * (rep = -1: the core operator only).  x_dev, hx_dev: device arrays [ncols][Ng] of `dtype`
 * (rmgtd_dtype), must not overlap.  Errors: RMGTD_EINVAL. */
int rmgtd_apply_h(rmgtd_ctx* ctx, const void* x_dev, void* hx_dev, int ncols, int dtype,
                  int rep);

/* Time-dependent external field E(t) of replica `rep` (Algorithm 1: the external potential
 * enters Omega through V_{j-1} + V_j, its values at both ends of the step).  Samples
 * E_xyz[j][q] = E_q(j dt), q = x, y, z (host, nsamp x 3 doubles, atomic units), with j
 * counted in completed steps of the context (t = j dt); E = 0 past the last sample.  A step
 * then propagates with Omega = -i dt (Hbar + sum_q ebar_q M_q), ebar = (E(t_j) + E(t_j + dt))/2:
 * the sign of the kick, so a field kappa delta(t) along q is the kick along q.  nsamp = 0
 * clears the replica's field.  rmgtd_energy reports the energy without the field's
 * interaction term.  The samples are copied and are not part of a checkpoint.  Errors:
 * RMGTD_EINVAL (replica, count, NULL or non-finite samples), RMGTD_ENOMEM, RMGTD_ESTATE (the
 * context belongs to a batch). */
int rmgtd_set_field(rmgtd_ctx* ctx, int rep, const double* E_xyz, int nsamp);

/* Delta kick of replica `rep` along axis q (0 = x, 1 = y, 2 = z):
 * P <- exp(-i kappa M_q) P exp(i kappa M_q) by the commutator expansion (Eq. 34 with a
 * delta envelope applied at t = 0+).  Errors: RMGTD_EINVAL, RMGTD_ENOTCONVERGED. */
int rmgtd_kick(rmgtd_ctx* ctx, int rep, int axis, double kappa);

/* Advance every replica by `nsteps` time steps of Algorithm 1.  `stats` (host, may be
 * NULL) receives nsteps * nrep entries, step-major.  Returns the first non-OK replica
 * status; on failure the state of the last completed step is kept. */
int rmgtd_step(rmgtd_ctx* ctx, int nsteps, rmgtd_stats* stats);

/* Result of the ground-state SCF (opt.ground_state_scf): iterations, final max|rho_out -
 * rho_in|, largest Ritz residual, and the N orbital energies (eps may be NULL).  Errors:
 * RMGTD_ESTATE when the context was created without it. */
int rmgtd_ground_state_info(rmgtd_ctx* ctx, int* iterations, double* drho, double* residual,
                            double* eps);

/* Dipole strength function of the kicked runs (Section 4: the spectrum is the sum of the
 * Fourier transforms of mu_x(t), mu_y(t), mu_z(t) of the runs kicked along x, y and z).
 * dipole: host [nq][nt] doubles, row q the dipole component along the kick of the run kicked
 * along q (by kappa), sampled at t_n = n dt.  With the trapezoid rule over the samples and an
 * exponential damping gamma >= 0 (Lorentzian lines):
 *   S(omega_w) = -(2 omega_w / (pi kappa nq)) sum_q sum_n w_n dt (d_q(t_n) - d_q(0))
 *                e^{-gamma t_n} sin(omega_w t_n),
 * i.e. (2 omega / pi) Im alpha(omega), alpha = -(1/kappa) FT(d - d(0)), whose integral over
 * omega > 0 is the electron count in a complete basis (sum rule).  omega: host [nw]; S: host
 * [nw] output.  Runs on the current device in float64 (one warp per frequency), allocating
 * and freeing its own device buffers; synchronous.  1 <= nq <= 64, 1 <= nw <= 2^24.
 * Errors: RMGTD_EINVAL (NULL pointers, sizes, dt <= 0, kappa = 0, gamma < 0), RMGTD_ECUDA;
 * the message is read with rmgtd_last_error(NULL). */
int rmgtd_spectrum(const double* dipole, int nq, long nt, double dt, double kappa, double gamma,
                   const double* omega, int nw, double* S);

/* rho(r) of replica `rep` for the current P (host array of Ng doubles). */
int rmgtd_density(rmgtd_ctx* ctx, int rep, double* rho_host);

/* Electronic dipole d_q = Tr(Re(P) M_q), q = x, y, z, of replica `rep` (host double[3]). */
int rmgtd_dipole(rmgtd_ctx* ctx, int rep, double mu[3]);

/* Total energy Tr(Re P H_core) + 1/2 h^3 sum rho V_H + h^3 sum rho eps_xc + E_ion of
 * replica `rep` at the last density evaluation. */
int rmgtd_energy(rmgtd_ctx* ctx, int rep, double* E);

/* Copy an N x N matrix (rmgtd_matrix) of replica `rep` to / from host memory. */
int rmgtd_get_matrix(rmgtd_ctx* ctx, int which, int rep, double* host_out);
int rmgtd_set_matrix(rmgtd_ctx* ctx, int which, int rep, const double* host_in);

/* Hartree potential of a device density (Ng doubles) with the context's grid: solves
 * Lap_12 V = -4 pi rho with monopole + dipole ghost values by conjugate gradients to
 * poisson_tol, preconditioned as chosen by rmgtd_set_hartree_preconditioner (default: the
 * sine transform; the multigrid V-cycle where its tables do not fit).  vh_dev is used as
 * the initial guess.  Errors: RMGTD_ENOTCONVERGED. */
int rmgtd_hartree(rmgtd_ctx* ctx, const double* rho_dev, double* vh_dev);

/* LDA (Slater + PZ81) on n device points: vxc_dev, exc_dev receive V_xc and eps_xc. */
int rmgtd_xc(rmgtd_ctx* ctx, const double* rho_dev, double* vxc_dev, double* exc_dev,
             size_t n);

/* The mixed path's xc increment (Algorithm 1's density-functional update, with the fields
 * kept as float32 increments against the set-up state):
 * dvxc_dev[g] = V_xc(rho0_dev[g] + drho_dev[g]) - V_xc(rho0_dev[g]) for the LDA of rmgtd_xc,
 * on n device points (rho0 double, drho and the result float).  Evaluated in float32 arithmetic on the increment, so the error is a few
 * float32 units of the increment itself; points near the density floor or across r_s = 1 take
 * two float64 evaluations.  Arrays belong to the caller.  Errors: RMGTD_EINVAL. */
int rmgtd_xc_increment(rmgtd_ctx* ctx, const double* rho0_dev, const float* drho_dev,
                       float* dvxc_dev, size_t n);

/* Checkpoint / resume of the propagation state (t, step count, P, H_0, H_-1, V_H of every
 * replica) to a binary file.  rmgtd_load requires a context created for the same system. */
int rmgtd_save(rmgtd_ctx* ctx, const char* path);
int rmgtd_load(rmgtd_ctx* ctx, const char* path);

/* Simulation time and completed steps of the context. */
int rmgtd_time(rmgtd_ctx* ctx, double* t, long long* steps);

/* Phases of a time step reported by rmgtd_profile_read, in the paper's Table 1 names:
 * 0 commutator expansion ("ELDYN"), 1 density ("Rho"), 2 Hartree solve ("Vh"),
 * 3 exchange-correlation, 4 Hamiltonian update ("Hupdate"), 5 other (bookkeeping). */
#define RMGTD_NPHASES 6

/* Start (enable = 1) or stop per-phase timing with CUDA events recorded on the context's
 * stream around each phase of rmgtd_step; resets the phase totals and the launch count. */
int rmgtd_profile(rmgtd_ctx* ctx, int enable);

/* Accumulated milliseconds and calls per phase since the last rmgtd_profile call
 * (host arrays of RMGTD_NPHASES, may be NULL) and the number of kernels the library has
 * launched since then (for graph steps: kernel nodes executed, counting each iteration of
 * the device-side loops).  Phase times are recorded for host-driven steps only
 * (use_graph = 0): a captured step has no per-phase events.  Synchronises the stream. */
int rmgtd_profile_read(rmgtd_ctx* ctx, double* phase_ms, long long* phase_calls,
                       long long* launches);

/* Work counters of the Hartree solve since the last rmgtd_profile call, for host-driven and
 * graph steps alike: replica solves (Section 2.1's Poisson problem, one per replica per DFT
 * evaluation) and conjugate-gradient iterations summed over them.  Either pointer may be
 * NULL.  Synchronises the stream. */
int rmgtd_profile_counters(rmgtd_ctx* ctx, long long* hartree_solves,
                           long long* hartree_iterations);

/* ---- Launch autotuning and batched systems -------------------------------------------------
 * rmgtd_autotune times the launch alternatives of the mixed path's density (tensor-core CTAs
 * per SM), Hamiltonian update (tensor-core or SIMT kernel x CTAs per SM) and the persistent
 * Hartree solve (all SMs, 1/2 or 1/4 of them) on this context's shapes, on scratch outputs,
 * and keeps the fastest; the state is not changed, but later results may differ at rounding
 * level (other reduction orders).  choice (may be NULL) receives {density CTAs per SM, Gram
 * on tensor cores (0/1), Gram CTAs per SM, Hartree block divisor}.  Synchronises. */
int rmgtd_autotune(rmgtd_ctx* ctx, int choice[4]);

/* Set / read the launch configuration directly, in rmgtd_autotune's order: density CTAs per
 * SM in 1..4, Gram on tensor cores 0/1 (used when Ng is a multiple of 4, else the SIMT
 * kernel runs), Gram CTAs per SM in {1, 2, 4, 8} (the tensor-core kernel uses at most 2),
 * Hartree block divisor in {1, 2, 4}.  Out-of-range values: RMGTD_EINVAL, nothing changed;
 * a context in a batch: RMGTD_ESTATE.  Results may change at rounding level. */
int rmgtd_set_tuning(rmgtd_ctx* ctx, const int choice[4]);
int rmgtd_get_tuning(const rmgtd_ctx* ctx, int choice[4]);

/* Preconditioner of the Hartree conjugate-gradient solve (Section 2.2's Poisson problem with
 * the 12th-order operator of Eq. 2; both precisions).  The operator and the stopping test are
 * the same for both; only the iteration count and rounding differ.
 *   RMGTD_PRECOND_DST (default): the 3-D sine transform (DST-I) diagonalising the Toeplitz
 *     part of the 12th-order operator, applied in float32 -- used when its matrices and tiles
 *     fit in shared memory (lines up to ~100 points), else the multigrid V-cycle runs;
 *   RMGTD_PRECOND_MG: the float32 multigrid V-cycle of 7-point operators.
 * Other values: RMGTD_EINVAL, nothing changed; a context in a batch: RMGTD_ESTATE. */
#define RMGTD_PRECOND_DST 0
#define RMGTD_PRECOND_MG 1
int rmgtd_set_hartree_preconditioner(rmgtd_ctx* ctx, int kind);
/* The preconditioner the context's Hartree solves use now (*kind: RMGTD_PRECOND_DST when it
 * was chosen and its tables fit, else RMGTD_PRECOND_MG).  Errors: RMGTD_EINVAL (NULL). */
int rmgtd_get_hartree_preconditioner(rmgtd_ctx* ctx, int* kind);

/* Several contexts (different systems, each with its replicas) stepped by one CUDA graph per
 * time step, launched once per step on the contexts' common stream.  When every context has
 * an SM budget (rmgtd_options.sm_budget) their steps are captured on parallel branches of the
 * graph and run concurrently, each on its share of the SMs; otherwise back to back.  Budgets
 * that sum to more than the SM count are allowed but then the branches partly wait for one
 * another.  All contexts must use the same stream; attach the
 * learned seed and autotune before creating the batch.  While in a batch a context refuses
 * rmgtd_step, rmgtd_attach_net and rmgtd_autotune (RMGTD_ESTATE); other calls work.
 * Errors: RMGTD_EINVAL (NULL, repeated or already-batched contexts, different streams). */
typedef struct rmgtd_batch rmgtd_batch;
int rmgtd_batch_create(rmgtd_ctx* const* ctxs, int n, rmgtd_batch** out);
void rmgtd_batch_destroy(rmgtd_batch* batch);
/* nsteps steps of every context; stats (may be NULL) holds one array per context, each of
 * nsteps x nrep records (as rmgtd_step).  On a failed step the error names the context. */
int rmgtd_batch_step(rmgtd_batch* batch, int nsteps, rmgtd_stats* const* stats);

/* ---- Learned seed of the SCF loop (Algorithm 1's extrapolation) ---------------------------
 * The paper seeds each step's Hamiltonian SCF loop with H_1 = 2 H_0 - H_-1 = H[2 V_0 - V_-1].
 * An attached network adds dV = s_out * y to that potential, y = net(x) with features
 *   x[0] = rho_t / s_0,  x[1] = (rho_t - rho_{t-dt}) / s_1,  x[2] = (rho_t - 2 rho_{t-dt} + rho_{t-2dt}) / s_2,
 * i.e. H_1 += h^3 Phi^T diag(dV) Phi before the first pass.  The SCF loop still decides
 * convergence (H_thrs), so the converged step does not depend on the network; only the
 * number of passes does.  Network: four 3x3x3 cross-correlations with zero padding,
 * 3 -> 16 -> 16 -> 16 -> 1 channels, SiLU after the first three; bfloat16 weights, float32
 * biases and accumulation.  Parameters (float32, RMGTD_NET_PARAMS of them): per layer W
 * [cout][cin][kz][ky][kx] then b [cout].  Training target: (V_{t+dt} - 2 V_t + V_{t-dt}) / s_out
 * (V = V_H + V_xc of converged steps); loss = mean squared error over the points at least 4
 * from every face; Adam (beta1 0.9, beta2 0.999, eps 1e-8) on float32 master parameters.
 * A network is not thread-safe; do not train one while an attached context steps. */
typedef struct rmgtd_net rmgtd_net;
#define RMGTD_NET_PARAMS 15601

long long rmgtd_net_num_params(void);
/* Network with workspace for batches of up to max_batch samples on an nx x ny x nz grid, its
 * calls ordered on `stream` (cudaStream_t, NULL = legacy default).  Parameters start at 0
 * (the paper's seed), scales at 1.  Errors: RMGTD_EINVAL, RMGTD_ENOMEM. */
int rmgtd_net_create(int nx, int ny, int nz, int max_batch, void* stream, rmgtd_net** out);
void rmgtd_net_destroy(rmgtd_net* net);
/* Copy the float32 parameter vector in from / out to host memory; set resets Adam. */
int rmgtd_net_set_params(rmgtd_net* net, const float* theta_host);
int rmgtd_net_get_params(rmgtd_net* net, float* theta_host);
/* Feature scales s_0..s_2 and output scale s_out (positive, finite). */
int rmgtd_net_set_scales(rmgtd_net* net, const double in_scales[3], double out_scale);
int rmgtd_net_get_scales(rmgtd_net* net, double in_scales[3], double* out_scale);
/* Weight file of the network (host file IO): tag "RMGTDNET", uint32 version 1, uint32 0,
 * int64 parameter count, float64 scales s_0, s_1, s_2, s_out, then the float32 parameters,
 * little-endian.  save writes the current parameters and scales; load checks the tag,
 * version and count (RMGTD_EINVAL otherwise, or for non-finite values) and replaces both
 * (Adam restarts). */
int rmgtd_net_save(rmgtd_net* net, const char* path);
int rmgtd_net_load(rmgtd_net* net, const char* path);
/* One sample's features x_dev [3][Ng] (float32) from three float64 densities, and its target
 * t_dev [Ng] from three float64 potentials V_{t+dt}, V_t, V_{t-dt} (all device pointers). */
int rmgtd_net_features(rmgtd_net* net, const double* rho_t, const double* rho_tm1,
                       const double* rho_tm2, float* x_dev);
int rmgtd_net_targets(rmgtd_net* net, const double* v_tp1, const double* v_t, const double* v_tm1,
                      float* t_dev);
/* y_dev [batch][Ng] = net(x_dev [batch][3][Ng]) (device pointers); synchronises the stream. */
int rmgtd_net_forward(rmgtd_net* net, const float* x_dev, float* y_dev, int batch);
/* The same with the two 16 -> 16 layers on the tensor cores, activations rounded to
 * bfloat16 at their inputs (float32 accumulation): the form the propagation's predictor
 * uses.  Synchronises the stream. */
int rmgtd_net_forward_tc(rmgtd_net* net, const float* x_dev, float* y_dev, int batch);
/* Loss and gradient at the current parameters for targets t_dev [batch][Ng]; the gradient
 * stays on the device for rmgtd_net_adam and is copied to grad_host (RMGTD_NET_PARAMS
 * floats) when that is not NULL.  The grid needs interior points (every side > 8). */
int rmgtd_net_backward(rmgtd_net* net, const float* x_dev, const float* t_dev, int batch,
                       double* loss, float* grad_host);
/* One Adam step with learning rate lr from the last gradient. */
int rmgtd_net_adam(rmgtd_net* net, double lr);
/* Attach (net != NULL) or detach the learned seed; the network's grid must match the
 * context's and its max_batch must be >= nrep.  The density history restarts (no history:
 * rho_{t-dt} = rho_{t-2dt} = rho_t).  Errors: RMGTD_EINVAL. */
int rmgtd_attach_net(rmgtd_ctx* ctx, rmgtd_net* net);
/* Create a network on the context's grid and stream (max_batch = nrep), load the weight
 * file `path` (rmgtd_net_load) and attach it: the learned seed shipped with a run.  The
 * caller owns *net_out (detach with rmgtd_attach_net(ctx, NULL) before rmgtd_net_destroy).
 * Errors: those of the three calls; nothing is attached on failure. */
int rmgtd_surrogate_load(rmgtd_ctx* ctx, const char* path, rmgtd_net** net_out);

/* Fields of replica `rep` of the current state copied to a device array of Ng doubles:
 * which = 0 rho, 1 V_H + V_xc (of the last DFT evaluation). */
#define RMGTD_FIELD_RHO 0
#define RMGTD_FIELD_VHXC 1
int rmgtd_get_field(rmgtd_ctx* ctx, int which, int rep, double* dev_out);

/* Allocation-free Gram contraction  C = scale * A^T diag(w) B  (N x N, row-major) for two
 * orbital blocks A, B of n_orb columns of n_grid points each (orbital-major device arrays,
 * as in rmgtd_system.phi0), w (n_grid device doubles) or NULL for w = 1; c_dev receives
 * n_orb * n_orb doubles.  With A = B = Phi, w = V and scale = h^3 this is the Hamiltonian
 * update matrix; with w = x, y, z the dipole matrices; with w = NULL the overlap.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot allocate
 * device memory when they call -- code that runs while a stream is being captured into a
 * CUDA graph, hosts that own all device memory through their own arena, loops that cannot
 * take cudaMalloc's implicit synchronisation.  It allocates nothing: its scratch is a fixed
 * 8 MiB array of float64 inside the library (held on every GPU that loads the library until
 * the process exits), so n_orb must satisfy n_orb^2 <= 1048576 (n_orb <= 1024); larger sizes
 * return RMGTD_EINVAL.  The first call on a device looks up the array's address on that
 * device (make that first call before any stream capture); the address is looked up again
 * when the device's current CUDA context has changed since (after cudaDeviceReset or a
 * rebuilt primary context), so such a call, too, should come before any capture.  All calls
 * share the array:
 * calls whose work overlaps on the device race; serialise them on one stream.  Work is
 * enqueued on `stream` (cudaStream_t, NULL = default stream) and the call does not wait.
 * Errors (message through rmgtd_last_error(NULL)): RMGTD_EINVAL, RMGTD_ECUDA. */
int rmgtd_gram_noalloc(const double* a_dev, const double* b_dev, const double* w_dev,
                       int n_orb, long long n_grid, double scale, double* c_dev, void* stream);

/* Failure-detection diagnostic (no counterpart in the paper): launches one block per SM
 * that wait at a grid barrier on a counter of their own which block 0 never reaches, with
 * the wait limited to `polls` polls (1 .. 20000000) instead of the library's default limit,
 * and returns the status the waiting blocks recorded -- RMGTD_ETIMEOUT when the bounded wait
 * gave up, as every device-side wait of the library does -- in *status_out.  The context's
 * propagation state, its status word and its barrier counters are not touched.
 * Synchronises the stream.  Errors: RMGTD_EINVAL (polls out of range, NULL), RMGTD_ECUDA. */
int rmgtd_selftest_barrier_timeout(rmgtd_ctx* ctx, unsigned polls, int* status_out);

/* Message of the last error on `ctx` (thread-local message when ctx is NULL). */
const char* rmgtd_last_error(const rmgtd_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* RMGTD_H */
