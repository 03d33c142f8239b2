// Internal definitions shared by the translation units of librmgtd (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/rmgtd.h"

namespace rmgtd {

constexpr int kThreads = 256;
constexpr int kFdRadius = 6;             // 12th-order central stencil (Section 2.1, Eq. 2)
constexpr double kRhoFloor = 1e-14;      // LDA floor
constexpr unsigned kSpinLimit = 20000000u;  // bounded device-side waits (seconds)

// 12th-order second-derivative weights a_0..a_6 (Fornberg closed form, exact rationals).
__host__ __device__ inline double fd_coef(int m) {
  switch (m) {
    case 0: return -5369.0 / 1800.0;
    case 1: return 12.0 / 7.0;
    case 2: return -15.0 / 56.0;
    case 3: return 10.0 / 189.0;
    case 4: return -1.0 / 112.0;
    case 5: return 2.0 / 1925.0;
    case 6: return -1.0 / 16632.0;
  }
  return 0.0;
}

// Per-replica control block living in device memory.
struct RepCtl {
  int active;      // SCF loop still running for this replica in the current step
  int passes;      // DFT evaluations in the current step
  int terms_last;  // terms of the last commutator expansion
  int terms_max;
  int terms_sum;
  int status;      // rmgtd_status of the current step
  double H_err;    // last max|H_new - H_1|
};

// Per-replica state of the preconditioned CG Hartree solve.
struct PcgState {
  double rz[2];    // (r, z) of the previous iteration, double-buffered by `cur`
  double bb;       // (b, b)
  double rr;       // last (r, r)
  int cur;
  int it;
  int done;
  int status;
};

struct MgLevel {
  int nx, ny, nz;
  long n;
  double h;
  float* x;   // [nrep][n] iterate
  float* b;   // [nrep][n] right-hand side
  float* t;   // [nrep][n] sweep / residual scratch
};

struct Buffer {
  void* ptr;
  size_t bytes;
};

}  // namespace rmgtd

struct rmgtd_ctx {
  // sizes
  int nx = 0, ny = 0, nz = 0;
  long Ng = 0;
  int N = 0, nocc = 0, nvirt = 0, nrep = 1;
  double h = 0, h3 = 0;
  int hartree_xc = 1;
  double v_ext_omega = 0;
  rmgtd_options opt{};
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int coop_ok = 0;

  // host copies
  std::vector<double> f;
  double E_ion = 0;
  double t = 0;
  long long steps = 0;
  std::string err;

  // orbitals and potentials
  double* phi = nullptr;       // [N][Ng]
  float* phi32 = nullptr;      // [N][Ng] (mixed precision)
  // the same orbitals in 32-point tiles: [ceil(Ng/32)][Np][32] with Np = 32 ceil(N/32), zero
  // beyond N and Ng (allocated up to whole 128-point tiles), so that a 32-orbital x 32-point
  // block is 4 contiguous KB and a 128-point tile 16 (tensor cores)
  float* phi32t = nullptr;
  // the same orbitals as two bfloat16 planes (hi, lo) [2][Np_pl][Ngp_pl] (Np_pl = N rounded up
  // to 32, Ngp_pl = Ng rounded up to 64, zero beyond) for the orbital-tiled tensor-core
  // contractions (32 < N <= 256); NULL when those are not used
  __nv_bfloat16* phi_pl = nullptr;
  __nv_bfloat16* bt_pl = nullptr;  // [nrep][2][Np_pl][Np_pl] density-change matrix (transposed)
  int Np_pl = 0;
  long Ngp_pl = 0;
  alignas(64) unsigned char tm_pa[128] = {};   // planes, 64 x 64 boxes (density operand A)
  alignas(64) unsigned char tm_pb[128] = {};   // planes, 64 x Np_pl boxes (Gram operand B)
  alignas(64) unsigned char tm_bt[128] = {};   // density-change planes, 64 x 32 boxes
  int rho_pl_attr = 0, gram_pl_attr = 0;       // dynamic shared memory set for the kernels
  // anchors of the orbital-plane contractions (per replica, consistent pairs): the density is
  // formed as rho(Sa) + sum (S - Sa)_ij phi_i phi_j and the Hamiltonian as
  // Ha + h^3 Phi^T diag(V - Va) Phi, so the split products' rounding scales with the change
  // since the last completed step, not with the distance from the set-up state
  double* Sa = nullptr;       // [nrep][N*N] Re P of the anchor
  double* Ha = nullptr;       // [nrep][N*N] H of the anchor potential
  float* rho_a32 = nullptr;   // [nrep][Ng] rho(Sa) - rho_ref
  float* dv_a32 = nullptr;    // [nrep][Ng] V_Hxc of the anchor - vref
  double* vion = nullptr;      // [Ng] V_loc + V_ext
  double* rho_core = nullptr;  // [Ng] frozen core density (xc only), or NULL
  double* rho_xc_ref = nullptr;  // [Ng] rho_ref + rho_core: base of the mixed xc increment
  double* f_dev = nullptr;     // [N]

  // Kleinman-Bylander projectors as dense boxes
  int nproj = 0;
  int* pbox = nullptr;         // [nproj][6] x0,y0,z0,bx,by,bz
  long long* poff = nullptr;   // [nproj+1] offsets into pval
  double* pval = nullptr;      // box values (normalised)
  double* Ekb = nullptr;       // [nproj]
  double* kb_coef = nullptr;   // [2][ncols][nproj] projections (re, im)
  int kb_coef_cols = 0;
  std::vector<int> h_pbox;
  std::vector<long long> h_poff;
  std::vector<double> h_Ekb;

  // shared N x N matrices
  double* Hcore = nullptr;
  double* M = nullptr;         // [3][N*N]
  double* Smat = nullptr;
  double* Href = nullptr;      // H_core + h^3 Phi^T V_ref Phi (mixed reference)

  // replica N x N matrices [nrep][N*N]
  double *S0 = nullptr, *A0 = nullptr, *S1 = nullptr, *A1 = nullptr;
  double *H0 = nullptr, *Hm1 = nullptr, *H1 = nullptr, *Hnew = nullptr;
  double* dbuf = nullptr;      // [nrep][4][N*N] commutator-series work
  double* Sref = nullptr;      // [N*N] reference Re P for the mixed path (diag f)

  // grid fields [nrep][Ng]
  double *rho = nullptr, *vh = nullptr, *vxc = nullptr, *exc = nullptr, *vhxc = nullptr;
  double* rho_ref = nullptr;   // [Ng] density of Sref (mixed)
  float* rho_ref32 = nullptr;  // [Ng] rho_ref rounded to float32 (mixed xc increment)
  double* vref = nullptr;      // [Ng] reference V_Hxc (mixed)
  double* vh_ref = nullptr;    // [Ng] reference V_H (mixed)
  float* dv32 = nullptr;       // [nrep][Ng] V_Hxc - vref (mixed)
  float* dvh32 = nullptr;      // [nrep][Ng] V_H - vh_ref (mixed, Hartree correction unknown)
  float* dvh_prev32 = nullptr; // [nrep][Ng] dvh32 one step earlier (initial-guess history)
  float* dvh_prev2_32 = nullptr; // [nrep][Ng] dvh32 two steps earlier
  float* shat32 = nullptr;     // [nrep][Np][Np] float32 density-change matrix (mixed)
  double* vh_prev = nullptr;   // [nrep][Ng] V_H one step earlier (initial-guess history)
  double* vh_prev2 = nullptr;  // [nrep][Ng] V_H two steps earlier
  float *pcg32_r = nullptr, *pcg32_z = nullptr, *pcg32_p = nullptr,
        *pcg32_Ap = nullptr, *pcg32_Az = nullptr;   // [nrep][Ng] float32 CG vectors (mixed)
  float* drho32 = nullptr;     // [nrep][Ng] rho - rho_ref in float32 (mixed)
  float* ghost32 = nullptr;    // [4][Ng] float32 copy of the ghost response fields (mixed)
  int mixed = 0;               // mixed-precision step active (after set-up)
  int subspace_iters = 0;      // subspace SCF iterations done at set-up
  double subspace_err = 0;     // last max|P_new - P| of the subspace SCF

  // split-K partials of the Gram contractions
  double* gram_part = nullptr;
  size_t gram_part_elems = 0;

  // Hartree solve
  double *pcg_r = nullptr, *pcg_z = nullptr, *pcg_p = nullptr,
         *pcg_Ap = nullptr, *pcg_Az = nullptr;    // [nrep][Ng]
  unsigned* bar2 = nullptr;          // grid-barrier counter of the persistent Hartree solve
  int coop_attr_set[2] = {0, 0};     // persistent Hartree kernel configured (float64, float32)
  int coop_grid[2] = {0, 0};
  int rho_tc_attr = 0;               // tensor-core density kernel configured
  // launch choices (defaults, or measured by rmgtd_autotune)
  int tune_rho_blocks = 3;           // CTAs per SM of the tensor-core density kernel
  int tune_gram_tc = 1;              // mixed Gram on the tensor cores (1) or SIMT (0)
  int tune_gram_blocks = 2;          // CTAs per SM over the Gram's (pair, replica-group) units
  int tune_coop_div = 1;             // persistent Hartree solve on (SMs / div) blocks
  void* tune_x = nullptr;            // Hartree unknown redirected while timing (autotune)
  int gram_tc_attr = 0;              // tensor-core Gram kernel configured
  // tiled-TMA descriptors of the tensor-core Gram kernel (CUtensorMap, 128 bytes each): the
  // float32 orbitals, and the weight rows of the last call (pointer, rows)
  alignas(64) unsigned char tm_phi[128] = {};
  alignas(64) unsigned char tm_w[128] = {};
  int tm_phi_ok = 0;
  const void* tm_w_key = nullptr;
  int tm_w_rows = 0;
  double* red_part = nullptr;  // reduction partials
  int red_blocks = 0;                // blocks of the grid-stride reduction kernels
  int red_cap = 0;                   // capacity of one partial slot
  rmgtd::PcgState* pcg = nullptr;   // [nrep]
  double* ghost = nullptr;          // [4][Ng] ghost response fields G0, Gx, Gy, Gz
  std::vector<rmgtd::MgLevel> mg;   // multi-CTA levels (level 0 = fine grid)
  int mg_tail_level = -1;           // first level solved inside one CTA
  size_t mg_tail_smem = 0;
  float* mg_cinv = nullptr;         // inverse of the coarsest operator (tail, transposed), or NULL
  int mg_cinv_smem = 0;             // the persistent solve keeps mg_cinv in shared memory
  float* dst_tab = nullptr;         // sine-transform preconditioner: S_x, S_y, S_z, lx, ly, lz
  int hartree_precond = RMGTD_PRECOND_DST;
  void* mg_table = nullptr;         // device level table of the persistent solve

  // control
  rmgtd::RepCtl* ctl = nullptr;     // [nrep]
  rmgtd::RepCtl* ctl_host = nullptr;  // pinned host mirror
  unsigned int* bar = nullptr;      // grid-barrier counter
  unsigned long long* errslots = nullptr;  // [nrep][max_terms+1]
  unsigned long long* errbits = nullptr;   // [nrep] SCF error max
  int* status = nullptr;            // device-wide status word
  double* obs = nullptr;            // [nrep][8] observables
  double* obs_host = nullptr;       // pinned

  // counters and per-phase event timing
  long long launches = 0;
  int profile = 0;
  std::vector<cudaEvent_t> ev_pool;   // pairs (begin, end)
  std::vector<int> ev_phase;
  int ev_n = 0;
  double phase_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long phase_calls[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  // CUDA graph of one time step
  cudaGraphExec_t step_exec = nullptr;
  cudaGraph_t step_graph = nullptr;
  int in_batch = 0;             // stepped through an rmgtd_batch (own step calls refused)
  // mixed path: the float64 fields (rho unless a network reads it, V_H, V_xc, eps_xc, V_Hxc)
  // lag the float32 increments of the last pass until mixed_fields64 rebuilds them
  int fields_stale = 0;
  int eldyn_cluster = -1;           // cluster size of the commutator kernel (-1: not probed)
  int shat_fresh = 0;               // the last commutator launch also wrote shat32 for S1
  // multipole moments of drho from the tensor-core density kernel: [rep][4][blocks] per-CTA
  // partials (rho_mom_blocks = 0: not formed by the last density launch)
  double* rho_mom = nullptr;
  long rho_mom_cap = 0;
  int rho_mom_blocks = 0;

  // external field E(t) (rmgtd_set_field): samples E_r(j dt) per replica [nrep][fld_cap][3],
  // their counts, the step's mean [nrep][3]; step_dev counts completed steps on the device
  int fld_on = 0;
  int fld_cap = 0;
  double* fld_samples = nullptr;
  int* fld_nsamp = nullptr;
  double* fld_ebar = nullptr;   // [nrep][3] mean, then [nrep][6] end values E(t_k), E(t_k + dt)
  std::vector<std::vector<double>> fld_host;
  // non-orthogonal basis (opt.nonorthogonal): S^-1; the pass's S^-1 (Hbar + V) per replica;
  // second-order Magnus term (opt.magnus_order 2): D per replica; both: [nrep][N*N]
  double* Sinv = nullptr;
  double* Gm = nullptr;
  double* Dm = nullptr;
  double* Hm2 = nullptr;        // H two steps earlier (opt.seed_order 2), [nrep][N*N]
  float* hbar32 = nullptr;      // mixed path, N > 64: Hbar in float32 [nrep][N*N] and the
  float* dbuf32 = nullptr;      // float32 series terms [nrep][2][2][N*N] (the series' tail)
  double* Hx0 = nullptr;        // scratch [nrep][N*N] x 2: H_0 + V_0, H_1 + V_1 (Omega_2)
  double* Hx1 = nullptr;
  // propagation on the grid (opt.grid_basis): occupied orbitals [nrep][2][N][Ng] (planar
  // complex) and the series' sum, float64; potentials V_0, V_-1, V_1 [nrep][Ng];
  // the step's mean field [nrep][3]; active flags; Gram / Cholesky / inverse scratch [5][N*N];
  // observable partials
  double* gp_psi = nullptr;
  double* gp_psi1 = nullptr;
  double* gp_ht = nullptr;      // H_core psi scratch of the observables
  double* gp_v0 = nullptr;
  double* gp_vm1 = nullptr;
  double* gp_vm2 = nullptr;     // V_-2 (seed_order 2 only)
  double* gp_vh1 = nullptr;     // V_H at the start of the last two steps (the first Hartree
  double* gp_vh2 = nullptr;     // solve's guess is their quadratic extrapolation)
  int gp_vh_hist = 0;           // how many of them are set (0..2)
  double* gp_v1 = nullptr;
  double* gp_ebar = nullptr;
  int* gp_active = nullptr;
  double* gp_gram = nullptr;
  double* gp_zpart = nullptr;   // per-block partials of the small complex Gram
  double* gp_obs = nullptr;
  std::vector<double> gp_obs_host;
  void* gp_ta = nullptr;        // series terms in the path's precision (float64 / float32),
  void* gp_tb = nullptr;        // double-buffered [nrep][2][N][Ng]
  void* gp_vtot = nullptr;      // V_ion + Vbar + Ebar.q in that precision [nrep][Ng]
  int* gp_sact = nullptr;       // [3][nrep]: replicas whose series is still running, then
                                // each series' status and term count (set on the device)
  int gp_terms_hint = 0;        // terms of the last series (the next one's first batch)
  void* gp_coef = nullptr;      // KB projections of the current term, terms' precision
                                // [nrep][2][N][nproj]
  alignas(64) unsigned char gp_tm_a[128] = {};   // tensor maps of the two term buffers
  alignas(64) unsigned char gp_tm_b[128] = {};
  alignas(64) unsigned char gp_tm_0[128] = {};   // and of gp_psi0f (float32 terms)
  float* gp_psi0f = nullptr;    // float32 terms: the step's psi in float32 (the first term's
                                // input, and the density change's reference) [nrep][2][N][Ng]
  double* gp_rho0 = nullptr;    // float32 terms: rho of the step's psi [nrep][Ng]
  float* gp_f32occ = nullptr;   // float32 terms: the occupations f [N] in float32
  int gp_tma = 0;               // the term kernel streams its tiles by TMA
  int* gp_kb_row = nullptr;     // KB lists by grid point: CSR row offsets [Ng + 1],
  int* gp_kb_p = nullptr;       // projector index and E_p beta_p(r) of each entry (the
  void* gp_kb_w = nullptr;      // latter in the terms' precision)
  int* gp_kb_pt = nullptr;      // grid index of every projector-box entry [nval]
  void* gp_pv = nullptr;        // projector-box values beta_p in the terms' precision [nval]
  float* gp_acc = nullptr;      // float32 terms: the series' sum, hi then lo [2][nrep][2][N][Ng]
                                // (shares the observables' scratch gp_ht: never live together)
  long long gp_steps = 0;
  // ground state on the device (opt.ground_state_scf): orbital energies, SCF iterations,
  // final density change and largest Ritz residual
  std::vector<double> gs_eps;
  int gs_iters = 0;
  double gs_err = 0.0, gs_resid = 0.0;
  long long* step_dev = nullptr;

  // learned seed of the SCF loop (attached network; buffers allocated at attach)
  rmgtd_net* net = nullptr;
  float* net_x = nullptr;       // [nrep][3][Ng] features
  float* net_y = nullptr;       // [nrep][Ng] network output
  float* net_dv32 = nullptr;    // [nrep][Ng] predicted dV (mixed path)
  double* net_dv64 = nullptr;   // [nrep][Ng] predicted dV (float64 path)
  double* rho_h1 = nullptr;     // [nrep][Ng] rho one step earlier
  double* rho_h2 = nullptr;     // [nrep][Ng] rho two steps earlier
  double* rho_start = nullptr;  // [nrep][Ng] rho at the start of the current step
  cudaStream_t aux[3] = {nullptr, nullptr, nullptr};  // SCF body, CG body, top-level capture
  int capturing = 0;
  int* failed = nullptr;            // sticky: a step of the current rmgtd_step call failed
  int* done_steps = nullptr;        // steps completed in the current rmgtd_step call
  rmgtd::RepCtl* stats_dev = nullptr;  // [stats_cap][nrep]
  rmgtd::RepCtl* stats_host = nullptr; // pinned mirror
  int stats_cap = 0;
  // kernel counts of the captured step: top level and SCF-pass body; executions of the
  // body are counted on the device (kexec[0])
  int cap_top = 0, cap_scf = 0;
  long long graph_steps = 0;
  unsigned long long* kexec = nullptr;

  std::vector<rmgtd::Buffer> buffers;
};

namespace rmgtd {

// ---- error helpers -----------------------------------------------------------------
int set_error(rmgtd_ctx* ctx, int code, const std::string& msg);
int cuda_check(rmgtd_ctx* ctx, cudaError_t e, const char* what);
#define RMGTD_CUDA(ctx, call)                                  \
  do {                                                         \
    cudaError_t _e = (call);                                   \
    if (_e != cudaSuccess) return rmgtd::cuda_check(ctx, _e, #call); \
  } while (0)
#define RMGTD_LAUNCH(ctx, what)                                \
  do {                                                         \
    cudaError_t _e = cudaGetLastError();                       \
    if (_e != cudaSuccess) return rmgtd::cuda_check(ctx, _e, what); \
  } while (0)

void* dev_alloc(rmgtd_ctx* ctx, size_t bytes);

// Phases of one SCF pass (event timing when profiling is on).
enum Phase { PH_ELDYN = 0, PH_RHO = 1, PH_HARTREE = 2, PH_XC = 3, PH_HUPDATE = 4, PH_OTHER = 5 };
void ph_begin(rmgtd_ctx* ctx, int phase);
void ph_end(rmgtd_ctx* ctx);
int ph_flush(rmgtd_ctx* ctx);

// ---- device helpers ----------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of `v` (blockDim.x a multiple of 32, <= 1024); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    v = warp_sum(v);
  }
  return v;
}
__device__ __forceinline__ double block_max(double v, double* sh) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    v = warp_max(v);
  }
  return v;
}

// max of non-negative doubles via their IEEE bit patterns (NaN sorts above +inf).
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier for cooperative launches.  `count` is zeroed before the launch and
// only grows; `target` = gridDim.x * (number of this barrier, counting from 1).  Thread 0
// of each block arrives with a release reduction (the block barrier before it orders the
// block's writes ahead of it) and polls with acquire loads (the block barrier after it
// orders the block's later reads behind it).  The wait gives up after `limit` polls
// (kSpinLimit unless a diagnostic passes a smaller one) and records RMGTD_ETIMEOUT in
// *status; returns false then.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned target, int* status,
                                             unsigned limit = kSpinLimit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    unsigned spins = 0;
    while (ld_acquire_u32(count) < target) {
      if (++spins > limit) {
        atomicCAS(status, 0, (int)RMGTD_ETIMEOUT);
        ok = 0;
        break;
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

__host__ __device__ inline double axis_coord(int i, int n, double h) {
  return ((double)i - 0.5 * (double)(n - 1)) * h;
}

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// ---- launchers -------------------------------------------------------------------------
void dev_free(rmgtd_ctx* ctx, void* p);
double* kb_coef_buffer(rmgtd_ctx* ctx, int ncols);
// KB projections coef[(2 j) np + p] = h^3 <beta_p, x_j> of ncols real columns (F64 or F32)
int kb_project_cols(rmgtd_ctx* ctx, const void* x, int ncols, int dtype, double* coef);
// k_grid.cu
int launch_vion(rmgtd_ctx* ctx, const double* pos_dev, const double* Z_dev,
                const double* rc_dev, int natoms);
int build_projectors(rmgtd_ctx* ctx, const rmgtd_system* sys);
int apply_h_dev(rmgtd_ctx* ctx, const void* x, void* hx, int ncols, int dtype,
                const double* vextra);
// vh_mode: 0 = vh is an input; 1 = vh <- vh_ref + dvh32 (mixed step); 2 = vh is an input
// and dvh32 <- vh - vh_ref (mixed refresh).  dv32 (if given) <- V_H + V_xc - vref.
// with_core: the context's frozen core density (if any) is added to rho in the xc (grid
// fields of the context; not for the stand-alone rmgtd_xc)
int launch_lda(rmgtd_ctx* ctx, const double* rho, double* vh, int vh_mode, double* vxc,
               double* exc, double* vhxc, float* dv32, long n, const RepCtl* ctl, int nrep,
               long stride, int with_xc, bool with_core = true);
// Mixed pass: dv32 <- dvh32 + V_xc(rho_ref + drho32) - V_xc(rho_ref) in float32 arithmetic.
int launch_xc_mixed(rmgtd_ctx* ctx, const RepCtl* ctl, int nrep);
// dv[g] <- V_xc(rho0[g] + d[g]) - V_xc(rho0[g]) (the same float32 increment, stand-alone).
int launch_xc_increment(rmgtd_ctx* ctx, const double* rho0, const float* d, float* dv, long n);
// rho <- rho_ref + drho32 for every replica.
int rho_from_increment(rmgtd_ctx* ctx);
// k_subspace.cu
// out[r] = base[r * bstride] + scale * A^T diag(w_r) B (bstride 0: one base for all replicas)
int gram(rmgtd_ctx* ctx, const double* A, const double* B, const double* w, long wstride,
         int nw, double scale, const double* base, double* out, const double* prev,
         const RepCtl* ctl, int sym, unsigned long long* errbits, long bstride = 0);
int rho_dev(rmgtd_ctx* ctx, const double* S, double* rho, const RepCtl* ctl, int nrep);
int rho_dev_mixed(rmgtd_ctx* ctx, const double* S, double* rho, const RepCtl* ctl, int nrep);
// w_anchor (may be NULL, orbital-plane path only): the weight is w - w_anchor
int gram_mixed(rmgtd_ctx* ctx, const float* w, long wstride, int nw, double scale,
               const double* base, double* out, const RepCtl* ctl, unsigned long long* errbits,
               long bstride = 0, const float* w_anchor = nullptr);
int to_float(rmgtd_ctx* ctx, const double* in, float* out, long n);
// out = a + b on n points
int add_fields(rmgtd_ctx* ctx, const double* a, const double* b, double* out, long n);
// phi32t <- phi32 in 32-point tiles (layout above)
int tile_orbitals(rmgtd_ctx* ctx);
// febar (may be NULL): [nrep][3] field of the step, Hbar += sum_q febar[r][q] M_q
// D (may be NULL): [nreps][N*N] real antisymmetric Omega_2 / tau per replica (pre-offset like
// Ha), the series then multiplies by Hbar + i D
int eldyn(rmgtd_ctx* ctx, const double* Ha, const double* Hb, long hstride, double tau,
          const double* S0, const double* A0, double* S1, double* A1, const RepCtl* ctl_in,
          RepCtl* ctl_out, int rep0, int nreps,
          float* shat_out = nullptr, const double* febar = nullptr, const double* D = nullptr,
          bool f32_tail = false);
// k_magnus.cu: the non-orthogonal basis and the second-order Magnus term
// set-up of the non-orthogonal basis: Sinv = S^-1 and P_0 = L^-T diag(f) L^-1 for every replica
int nonorth_setup(rmgtd_ctx* ctx);
// per SCF pass, before the series: G = S^-1 (Hbar + V) into ctx->Gm (non-orthogonal basis) and
// D = (dt/12)[H_0 + V_0, H_1 + V_1] into ctx->Dm (Omega_2); *Ha/*Hb/*hstride/*febar/*D are the
// arguments the series then takes
int magnus_prepare(rmgtd_ctx* ctx, const double** Ha, const double** Hb, long* hstride,
                   const double** febar, const double** D);
// out_r = (Ha_r + Hb_r)/2 + sum_q febar[rep0 + r][q] M_q for nreps replicas (stride hstride)
int hbar_with_field(rmgtd_ctx* ctx, const double* Ha, const double* Hb, long hstride,
                    const double* febar, int rep0, int nreps, double* out);
// G = S^-1 M_axis into ctx->Gm for a kick in the non-orthogonal basis
int nonorth_kick_matrix(rmgtd_ctx* ctx, int axis);
// k_gridprop.cu: propagation of the occupied orbitals on the grid (opt.grid_basis)
int gridprop_setup(rmgtd_ctx* ctx);
int gridprop_kick(rmgtd_ctx* ctx, int rep, int axis, double kappa);
// one time step of every replica; st (may be NULL): nrep entries
int gridprop_step(rmgtd_ctx* ctx, rmgtd_stats* st);
int gridprop_observables(rmgtd_ctx* ctx);
void gridprop_read(const rmgtd_ctx* ctx, int rep, double* d3, double* E, double* ne);
// the step's mean field ebar from the samples (no-op without a field)
int field_begin(rmgtd_ctx* ctx);
int step_begin(rmgtd_ctx* ctx);
// step_begin and the quadratic extrapolation of the Hartree guess in one launch
int step_begin_extrapolate(rmgtd_ctx* ctx);
int scf_control(rmgtd_ctx* ctx, const unsigned long long* errbits,
                cudaGraphConditionalHandle cond, int use_cond);
// launches counted while the SCF body was captured, minus the Hartree-iteration body
int step_end(rmgtd_ctx* ctx);
int observables(rmgtd_ctx* ctx);
int subspace_update(rmgtd_ctx* ctx, double alpha, double* err_dev);
int orthonormalize(rmgtd_ctx* ctx);
// X <- L^-1 X for N columns of length Ng (L lower, row-major); work: N * Ng doubles
int forward_subst(rmgtd_ctx* ctx, int N, const double* L, double* X, double* work);
// k_groundstate.cu: SCF ground state of the Kohn-Sham orbitals from ctx->phi (orthonormal),
// replacing ctx->phi by the N lowest eigenvectors of H[rho] (opt.ground_state_scf > 0)
int ground_state_scf(rmgtd_ctx* ctx);
// in-place lower Cholesky factor of the N x N matrix S (one block; status <- EINVAL when a
// pivot is not positive)
__global__ void k_cholesky(int N, double* __restrict__ S, int* status);
// k_poisson.cu
int setup_multigrid(rmgtd_ctx* ctx);
int poisson_red_cap(int num_sms, int red_blocks);
// Hartree solve of every active replica in one cooperative launch; f32 = 1: float32
// correction solve of the mixed path (reads drho32, writes dvh32)
// xc_fuse (float32 path): the kernel's closing phase also writes dv32 = dV_H + dV_xc
int hartree_coop(rmgtd_ctx* ctx, const double* rho, double* vh, const RepCtl* ctl, int zero_bc,
                 int nrep, int f32, int xc_fuse = 0);
int hartree_reset_history(rmgtd_ctx* ctx);
int hartree_precond_in_use(rmgtd_ctx* ctx);
// k_tc.cu
int rho_tc(rmgtd_ctx* ctx, double* rho, float* drho, const RepCtl* ctl, int nrep);
int gram_tc(rmgtd_ctx* ctx, const float* w, int nw, float* part, int nsplit, int chunk,
            const RepCtl* ctl);
// k_contract.cu (orbital planes, 32 < N <= 256): set-up, and the two contractions; the latter
// return 1 when the planes are not set up (the caller then uses the other kernels)
int planes_setup(rmgtd_ctx* ctx);
// anchors <- the set-up reference state (all replicas)
int planes_anchor_reset(rmgtd_ctx* ctx);
// after a completed step (same condition as k_step_end): Sa <- S0, Ha <- H0, rho_a <- drho,
// Va <- dV of every replica
int planes_anchor_update(rmgtd_ctx* ctx);
int rho_planes(rmgtd_ctx* ctx, const double* S, double* rho, float* drho, const RepCtl* ctl,
               int nrep);
// w_anchor (may be NULL): the weight is w - w_anchor
int gram_planes(rmgtd_ctx* ctx, const float* w, const float* w_anchor, int nw, float* part,
                int nsplit, int chunk, const RepCtl* ctl);
int conv16_tc(int nx, int ny, int nz, int B, const float* x, const __nv_bfloat16* W,
              const float* bias, float* y, int silu, int* status, int num_sms, cudaStream_t s);
// k_surrogate.cu
int net_forward_on(rmgtd_net* n, const float* x, float* y, int batch, cudaStream_t s, bool keep_pre,
                   bool tc_middle, int* status);
int net_batch_cap(const rmgtd_net* n);
long net_grid_points(const rmgtd_net* n, int* nx, int* ny, int* nz);
int net_predict(rmgtd_ctx* ctx);
int net_history_shift(rmgtd_ctx* ctx);
int net_history_reset(rmgtd_ctx* ctx);

}  // namespace rmgtd
