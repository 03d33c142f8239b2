// The C ABI of include/rmgtd.h: context set-up (Algorithm 1's set-up), the time loop
// (Algorithm 1's time loop), kicks, observables, checkpoints.  Host code only orchestrates launches on
// the context's stream; every arithmetic step of the propagation runs in the kernels of
// k_grid.cu, k_subspace.cu and k_poisson.cu.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <string>

#include "rmgtd_internal.cuh"

static thread_local std::string g_last_error;

namespace rmgtd {

int set_error(rmgtd_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  g_last_error = msg;
  return code;
}

int cuda_check(rmgtd_ctx* ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return set_error(ctx, RMGTD_ENOMEM, m);
  return set_error(ctx, RMGTD_ECUDA, m);
}

void* dev_alloc(rmgtd_ctx* ctx, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (ctx->opt.alloc) {
    p = ctx->opt.alloc(bytes, (void*)ctx->stream, ctx->opt.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    p = nullptr;
  }
  if (p) ctx->buffers.push_back(Buffer{p, bytes});
  return p;
}

void dev_free(rmgtd_ctx* ctx, void* p) {
  if (!p) return;
  for (size_t i = 0; i < ctx->buffers.size(); ++i) {
    if (ctx->buffers[i].ptr == p) {
      if (ctx->opt.free)
        ctx->opt.free(p, ctx->opt.alloc_user);
      else
        cudaFree(p);
      ctx->buffers.erase(ctx->buffers.begin() + i);
      return;
    }
  }
}

double* kb_coef_buffer(rmgtd_ctx* ctx, int ncols) {
  if (ncols > ctx->kb_coef_cols) {
    cudaStreamSynchronize(ctx->stream);
    dev_free(ctx, ctx->kb_coef);
    ctx->kb_coef = (double*)dev_alloc(ctx, sizeof(double) * 2 * (size_t)ctx->nproj * ncols);
    ctx->kb_coef_cols = ctx->kb_coef ? ncols : 0;
  }
  return ctx->kb_coef;
}

// ---- per-phase event timing ---------------------------------------------------------------
constexpr int kEvPairs = 512;

void ph_begin(rmgtd_ctx* ctx, int phase) {
  if (!ctx->profile || ctx->capturing) return;
  if (ctx->ev_n >= kEvPairs) ph_flush(ctx);
  cudaEventRecord(ctx->ev_pool[2 * ctx->ev_n], ctx->stream);
  ctx->ev_phase[ctx->ev_n] = phase;
}

void ph_end(rmgtd_ctx* ctx) {
  if (!ctx->profile || ctx->capturing) return;
  cudaEventRecord(ctx->ev_pool[2 * ctx->ev_n + 1], ctx->stream);
  ctx->ev_n += 1;
}

int ph_flush(rmgtd_ctx* ctx) {
  if (ctx->ev_n == 0) return RMGTD_OK;
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < ctx->ev_n; ++i) {
    float ms = 0.f;
    RMGTD_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_pool[2 * i], ctx->ev_pool[2 * i + 1]));
    ctx->phase_ms[ctx->ev_phase[i]] += ms;
    ctx->phase_calls[ctx->ev_phase[i]] += 1;
  }
  ctx->ev_n = 0;
  return RMGTD_OK;
}

// ---- small elementwise kernels ------------------------------------------------------------
__global__ void k_coords(int nx, int ny, int nz, double h, double* __restrict__ q) {
  const long Ng = (long)nx * ny * nz;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng;
       g += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(g % nx), iy = (int)((g / nx) % ny), iz = (int)(g / ((long)nx * ny));
    q[g] = axis_coord(ix, nx, h);
    q[Ng + g] = axis_coord(iy, ny, h);
    q[2 * Ng + g] = axis_coord(iz, nz, h);
  }
}

__global__ void k_symmetrize(int N, const double* __restrict__ in, double* __restrict__ out) {
  const long NN = (long)N * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < NN;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    out[e] = 0.5 * (in[e] + in[(long)j * N + i]);
  }
}

__global__ void k_diag_init(int N, int nrep, const double* __restrict__ f, double* __restrict__ S,
                            double* __restrict__ A) {
  const long NN = (long)N * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < NN * nrep;
       e += (long)gridDim.x * blockDim.x) {
    const long l = e % NN;
    const int i = (int)(l / N), j = (int)(l % N);
    S[e] = (i == j) ? f[i] : 0.0;
    A[e] = 0.0;
  }
}

__global__ void k_set_active(RepCtl* ctl, int nrep, int v) {
  if (threadIdx.x < nrep) {
    ctl[threadIdx.x].active = v;
    ctl[threadIdx.x].status = 0;
  }
}

__global__ void k_ion_energy(int natoms, const double* __restrict__ pos, const double* __restrict__ Z,
                             const double* __restrict__ rc, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  const long npair = (long)natoms * natoms;
  for (long e = threadIdx.x; e < npair; e += blockDim.x) {
    const int a = (int)(e / natoms), b = (int)(e % natoms);
    if (b >= a) continue;
    const double dx = pos[3 * a] - pos[3 * b], dy = pos[3 * a + 1] - pos[3 * b + 1],
                 dz = pos[3 * a + 2] - pos[3 * b + 2];
    const double R = sqrt(dx * dx + dy * dy + dz * dz);
    const double sg = sqrt(rc[a] * rc[a] + rc[b] * rc[b]);
    s += Z[a] * Z[b] * erf(R / sg) / R;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

// ---- CUDA-graph helpers -----------------------------------------------------------------------
// Add a while-loop node at the current capture position of ctx->stream; returns its body
// graph and handle.  The handle starts each launch of the node at 1 (the body runs at least
// once) and the body's last kernel sets it.
// Handle for a while loop that will be added to the graph being captured on ctx->stream.
// The top-level loop uses default value 1 (reset at every launch of the step graph); a
// nested loop gets no default and is armed by a kernel just before it.
static int new_handle(rmgtd_ctx* ctx, cudaGraphConditionalHandle* h, bool with_default) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  RMGTD_CUDA(ctx, cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
  if (cs != cudaStreamCaptureStatusActive) return set_error(ctx, RMGTD_ECUDA, "stream not capturing");
  if (with_default) {
    RMGTD_CUDA(ctx, cudaGraphConditionalHandleCreate(h, g, 1, cudaGraphCondAssignDefault));
  } else {
    RMGTD_CUDA(ctx, cudaGraphConditionalHandleCreate(h, g, 0, 0));
  }
  return RMGTD_OK;
}

// Add a while-loop node driven by `h` at the current capture position of ctx->stream and
// return its body graph.
static int add_while(rmgtd_ctx* ctx, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  RMGTD_CUDA(ctx, cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return set_error(ctx, RMGTD_ECUDA, "stream not capturing");
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  RMGTD_CUDA(ctx, cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  *body = p.conditional.phGraph_out[0];
  RMGTD_CUDA(ctx, cudaStreamUpdateCaptureDependencies(ctx->stream, &node, nullptr, 1,
                                                      cudaStreamSetCaptureDependencies));
  return RMGTD_OK;
}


// ---- one density-functional evaluation: H_1 <- DFT(rho(P)) (Algorithm 1's update) ------------
// S: Re P per replica.  Writes rho, vh, vxc, exc, vhxc and H1 (in place) for active
// replicas and folds max|H_new - H_1| into errbits.
int dft_eval(rmgtd_ctx* ctx, const double* S, const RepCtl* ctl, unsigned long long* errbits) {
  const int nrep = ctx->nrep;
  const int mixed = ctx->mixed;
  ph_begin(ctx, PH_RHO);
  // the mixed pass keeps the density as its float32 increment; the float64 copy is written
  // only for an attached network, whose features read it
  int rc = mixed ? rho_dev_mixed(ctx, S, ctx->net ? ctx->rho : nullptr, ctl, nrep)
                 : rho_dev(ctx, S, ctx->rho, ctl, nrep);
  ph_end(ctx);
  if (rc) return rc;
  if (ctx->hartree_xc) {
    ph_begin(ctx, PH_HARTREE);
    // mixed: the solve's closing phase also forms dV = dV_H + dV_xc (no separate xc pass),
    // and it takes the multipole moments from the density kernel when that formed them
    rc = hartree_coop(ctx, ctx->rho, ctx->vh, ctl, 0, nrep, mixed, mixed);
    ctx->rho_mom_blocks = 0;
    ph_end(ctx);
    if (rc) return rc;
  }
  ph_begin(ctx, PH_XC);
  if (mixed) {
    if (!ctx->hartree_xc) rc = launch_xc_mixed(ctx, ctl, nrep);
    ctx->fields_stale = 1;
  } else {
    rc = launch_lda(ctx, ctx->rho, ctx->hartree_xc ? ctx->vh : nullptr, 0, ctx->vxc, ctx->exc,
                    ctx->vhxc, nullptr, ctx->Ng, ctl, nrep, ctx->Ng, ctx->hartree_xc);
  }
  ph_end(ctx);
  if (rc) return rc;
  if (errbits)
    RMGTD_CUDA(ctx, cudaMemsetAsync(errbits, 0, sizeof(unsigned long long) * nrep, ctx->stream));
  ph_begin(ctx, PH_HUPDATE);
  if (mixed && ctx->Ha)   // orbital planes: H = Ha + h^3 Phi^T diag(dV - dVa) Phi per replica
    rc = gram_mixed(ctx, ctx->dv32, ctx->Ng, nrep, ctx->h3, ctx->Ha, ctx->H1, ctl, errbits,
                    (long)ctx->N * ctx->N, ctx->dv_a32);
  else if (mixed)
    rc = gram_mixed(ctx, ctx->dv32, ctx->Ng, nrep, ctx->h3, ctx->Href, ctx->H1, ctl, errbits);
  else
    rc = gram(ctx, ctx->phi, ctx->phi, ctx->vhxc, ctx->Ng, nrep, ctx->h3, ctx->Hcore, ctx->H1,
              errbits ? ctx->H1 : nullptr, ctl, 1, errbits);
  ph_end(ctx);
  return rc;
}

// Rebuild the float64 fields of the mixed path from the float32 increments of the last pass:
// rho = rho_ref + drho, V_H = V_H,ref + dV_H, then V_xc, eps_xc, V_Hxc by the float64 LDA.
int mixed_fields64(rmgtd_ctx* ctx) {
  if (!ctx->mixed || !ctx->fields_stale) return RMGTD_OK;
  int rc = rho_from_increment(ctx);
  if (rc) return rc;
  rc = launch_lda(ctx, ctx->rho, ctx->hartree_xc ? ctx->vh : nullptr, ctx->hartree_xc ? 1 : 0,
                  ctx->vxc, ctx->exc, ctx->vhxc, nullptr, ctx->Ng, nullptr, ctx->nrep, ctx->Ng,
                  ctx->hartree_xc);
  if (rc) return rc;
  ctx->fields_stale = 0;
  return RMGTD_OK;
}

// Refresh rho / V_H / V_xc / eps_xc from the current P_0 of every replica (no H update),
// in float64 (kicks, loads, set_matrix); in the mixed path the float32 corrections are
// re-derived from the float64 fields.
int refresh_fields(rmgtd_ctx* ctx) {
  int rc = rho_dev(ctx, ctx->S0, ctx->rho, nullptr, ctx->nrep);
  if (rc) return rc;
  if (ctx->hartree_xc) {
    rc = hartree_coop(ctx, ctx->rho, ctx->vh, nullptr, 0, ctx->nrep, 0);
    if (rc) return rc;
  }
  rc = launch_lda(ctx, ctx->rho, ctx->hartree_xc ? ctx->vh : nullptr,
                  (ctx->mixed && ctx->hartree_xc) ? 2 : 0, ctx->vxc, ctx->exc, ctx->vhxc,
                  ctx->mixed ? ctx->dv32 : nullptr, ctx->Ng, nullptr, ctx->nrep, ctx->Ng,
                  ctx->hartree_xc);
  if (rc) return rc;
  ctx->fields_stale = 0;
  if (ctx->net) {
    rc = net_history_reset(ctx);
    if (rc) return rc;
  }
  return hartree_reset_history(ctx);
}

static int check_status(rmgtd_ctx* ctx, const char* where) {
  int st = 0;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(&ctx->ctl_host[ctx->nrep], ctx->status, sizeof(int),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  memcpy(&st, &ctx->ctl_host[ctx->nrep], sizeof(int));
  if (st != 0) {
    char buf[160];
    snprintf(buf, sizeof(buf), "%s: device status %d", where, st);
    return set_error(ctx, st, buf);
  }
  return RMGTD_OK;
}

// Diagnostic of the bounded waits: every block but block 0 waits at one grid barrier that
// block 0 never reaches, giving up after `limit` polls (status[0] <- RMGTD_ETIMEOUT).
__global__ void k_barrier_timeout_probe(unsigned* count, int* status, unsigned limit) {
  if (blockIdx.x == 0) return;
  grid_barrier(count, gridDim.x, status, limit);
}

}  // namespace rmgtd

using namespace rmgtd;

extern "C" {

void rmgtd_default_options(rmgtd_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->dt = 0.05;
  o->H_thrs = 1e-7;
  o->dP_thrs = 1e-10;
  o->max_scf = 50;
  o->max_terms = 200;
  o->precision = RMGTD_PREC_FP64;
  o->nrep = 1;
  o->orthonormalize = 1;
  o->poisson_tol = 1e-12;
  o->poisson_max_iter = 200;
  o->use_graph = 1;
  o->subspace_scf = 0;
  o->subspace_mix = 0.3;
  o->subspace_tol = 1e-10;
  o->magnus_order = 1;
  o->nonorthogonal = 0;
  o->grid_basis = 0;
  o->ground_state_scf = 0;
  o->ground_state_tol = 1e-8;
  o->seed_order = 1;
  o->sm_budget = 0;
}

const char* rmgtd_last_error(const rmgtd_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  return g_last_error.c_str();
}

void rmgtd_destroy(rmgtd_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
  for (auto& b : ctx->buffers) {
    if (ctx->opt.free)
      ctx->opt.free(b.ptr, ctx->opt.alloc_user);
    else
      cudaFree(b.ptr);
  }
  ctx->buffers.clear();
  if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
  if (ctx->obs_host) cudaFreeHost(ctx->obs_host);
  if (ctx->stats_host) cudaFreeHost(ctx->stats_host);
  for (auto& e : ctx->ev_pool) cudaEventDestroy(e);
  for (int i = 0; i < 3; ++i)
    if (ctx->aux[i]) cudaStreamDestroy(ctx->aux[i]);
  delete ctx;
}

static int create_impl(const rmgtd_system* sys, const rmgtd_options* opt, rmgtd_ctx* ctx) {
  ctx->opt = *opt;
  ctx->stream = (cudaStream_t)opt->stream;
  ctx->nx = sys->nx;
  ctx->ny = sys->ny;
  ctx->nz = sys->nz;
  ctx->Ng = (long)sys->nx * sys->ny * sys->nz;
  ctx->h = sys->h;
  ctx->h3 = sys->h * sys->h * sys->h;
  ctx->nocc = sys->nocc;
  ctx->nvirt = sys->nvirt;
  ctx->N = sys->nocc + sys->nvirt;
  ctx->nrep = opt->nrep;
  ctx->hartree_xc = sys->hartree_xc ? 1 : 0;
  ctx->v_ext_omega = sys->v_ext_omega;
  const int N = ctx->N;
  const long Ng = ctx->Ng;
  const long NN = (long)N * N;
  const int nrep = ctx->nrep;

  int dev = 0;
  RMGTD_CUDA(ctx, cudaGetDevice(&dev));
  cudaDeviceProp prop;
  RMGTD_CUDA(ctx, cudaGetDeviceProperties(&prop, dev));
  ctx->num_sms = prop.multiProcessorCount;
  if (opt->sm_budget > 0)   // every grid, persistent kernels included, sized to this share
    ctx->num_sms = std::min(ctx->num_sms, opt->sm_budget);
  ctx->coop_ok = prop.cooperativeLaunch;
  if (!ctx->coop_ok) return set_error(ctx, RMGTD_ECUDA, "device lacks cooperative launch");
  // blocks of the grid-stride reduction kernels: about one point per thread up to 2048
  ctx->red_blocks = 2 * ctx->num_sms;
  ctx->red_cap = poisson_red_cap(ctx->num_sms, ctx->red_blocks);

  ctx->f.assign(N, 0.0);
  for (int i = 0; i < N; ++i) ctx->f[i] = sys->f ? sys->f[i] : (i < sys->nocc ? 2.0 : 0.0);

  auto A = [&](size_t bytes) { return dev_alloc(ctx, bytes); };
  const size_t gsz = sizeof(double) * Ng, msz = sizeof(double) * NN;
  ctx->phi = (double*)A(gsz * N);
  ctx->vion = (double*)A(gsz);
  ctx->f_dev = (double*)A(sizeof(double) * N);
  ctx->Hcore = (double*)A(msz);
  ctx->M = (double*)A(3 * msz);
  ctx->Smat = (double*)A(msz);
  ctx->S0 = (double*)A(msz * nrep);
  ctx->A0 = (double*)A(msz * nrep);
  ctx->S1 = (double*)A(msz * nrep);
  ctx->A1 = (double*)A(msz * nrep);
  ctx->H0 = (double*)A(msz * nrep);
  ctx->Hm1 = (double*)A(msz * nrep);
  if (opt->seed_order == 2) ctx->Hm2 = (double*)A(msz * nrep);
  if (opt->precision == RMGTD_PREC_MIXED && !opt->grid_basis && N > 64) {
    ctx->hbar32 = (float*)A(sizeof(float) * NN * nrep);
    ctx->dbuf32 = (float*)A(sizeof(float) * 4 * NN * nrep);
  }
  ctx->H1 = (double*)A(msz * nrep);
  ctx->dbuf = (double*)A(4 * msz * nrep);
  ctx->rho = (double*)A(gsz * nrep);
  ctx->vh = (double*)A(gsz * nrep);
  ctx->vh_prev = (double*)A(gsz * nrep);
  ctx->vh_prev2 = (double*)A(gsz * nrep);
  ctx->vxc = (double*)A(gsz * nrep);
  ctx->exc = (double*)A(gsz * nrep);
  ctx->vhxc = (double*)A(gsz * nrep);
  ctx->pcg_r = (double*)A(gsz * nrep);
  ctx->pcg_z = (double*)A(gsz * nrep);
  ctx->pcg_p = (double*)A(gsz * nrep);
  ctx->pcg_Ap = (double*)A(gsz * nrep);
  ctx->pcg_Az = (double*)A(gsz * nrep);
  ctx->bar2 = (unsigned*)A(sizeof(unsigned));
  ctx->red_part = (double*)A(sizeof(double) * (size_t)nrep * 8 * ctx->red_cap);
  ctx->pcg = (PcgState*)A(sizeof(PcgState) * nrep);
  ctx->ctl = (RepCtl*)A(sizeof(RepCtl) * nrep);
  ctx->bar = (unsigned*)A(sizeof(unsigned));
  ctx->errslots = (unsigned long long*)A(sizeof(unsigned long long) * (size_t)nrep * (opt->max_terms + 1));
  ctx->errbits = (unsigned long long*)A(sizeof(unsigned long long) * nrep);
  ctx->status = (int*)A(sizeof(int));
  ctx->obs = (double*)A(sizeof(double) * 8 * nrep);
  ctx->failed = (int*)A(sizeof(int));
  ctx->kexec = (unsigned long long*)A(4 * sizeof(unsigned long long));
  ctx->done_steps = (int*)A(sizeof(int));
  ctx->step_dev = (long long*)A(sizeof(long long));
  ctx->fld_ebar = (double*)A(sizeof(double) * 9 * nrep);
  // Omega's scratch: Hbar + V of a field step, H_0 + V_0 / H_1 + V_1 of Omega_2
  ctx->Hx0 = (double*)A(msz * nrep);
  if (opt->nonorthogonal || opt->magnus_order == 2) ctx->Hx1 = (double*)A(msz * nrep);
  if (opt->nonorthogonal) {
    ctx->Sinv = (double*)A(msz);
    ctx->Gm = (double*)A(msz * nrep);
  }
  if (opt->magnus_order == 2) ctx->Dm = (double*)A(msz * nrep);
  ctx->fld_nsamp = (int*)A(sizeof(int) * nrep);
  ctx->fld_host.assign(nrep, std::vector<double>());
  ctx->stats_cap = 256;
  ctx->stats_dev = (RepCtl*)A(sizeof(RepCtl) * ctx->stats_cap * nrep);
  {
    const long per = std::max(3, nrep) * NN;
    const long want = per * 4L * ctx->num_sms;
    const long cap = std::max<long>(per, 64L << 20);
    ctx->gram_part_elems = (size_t)std::min(want, cap);
    ctx->gram_part = (double*)A(sizeof(double) * ctx->gram_part_elems);
  }
  for (auto& b : ctx->buffers)
    if (!b.ptr) return set_error(ctx, RMGTD_ENOMEM, "device allocation failed");
  if (!ctx->phi || !ctx->gram_part || !ctx->pcg_Ap || !ctx->dbuf || !ctx->errslots)
    return set_error(ctx, RMGTD_ENOMEM, "device allocation failed");
  RMGTD_CUDA(ctx, cudaMallocHost((void**)&ctx->ctl_host, sizeof(RepCtl) * (nrep + 2)));
  RMGTD_CUDA(ctx, cudaMallocHost((void**)&ctx->obs_host, sizeof(double) * 8 * nrep));
  RMGTD_CUDA(ctx, cudaMallocHost((void**)&ctx->stats_host, sizeof(RepCtl) * ctx->stats_cap * nrep));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->failed, 0, sizeof(int), ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->step_dev, 0, sizeof(long long), ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->fld_ebar, 0, sizeof(double) * 9 * nrep, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->fld_nsamp, 0, sizeof(int) * nrep, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->kexec, 0, 4 * sizeof(unsigned long long), ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->vh, 0, gsz * nrep, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->ctl, 0, sizeof(RepCtl) * nrep, ctx->stream));

  // orbitals, occupations, atoms
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->phi, sys->phi0, gsz * N, cudaMemcpyHostToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->f_dev, ctx->f.data(), sizeof(double) * N,
                                  cudaMemcpyHostToDevice, ctx->stream));
  const int na = sys->natoms;
  double* pos_d = (double*)A(sizeof(double) * 3 * std::max(na, 1));
  double* Z_d = (double*)A(sizeof(double) * std::max(na, 1));
  double* rc_d = (double*)A(sizeof(double) * std::max(na, 1));
  double* eion_d = (double*)A(sizeof(double));
  if (!pos_d || !Z_d || !rc_d || !eion_d) return set_error(ctx, RMGTD_ENOMEM, "atom arrays");
  if (na > 0) {
    RMGTD_CUDA(ctx, cudaMemcpyAsync(pos_d, sys->pos, sizeof(double) * 3 * na, cudaMemcpyHostToDevice, ctx->stream));
    RMGTD_CUDA(ctx, cudaMemcpyAsync(Z_d, sys->Z, sizeof(double) * na, cudaMemcpyHostToDevice, ctx->stream));
    RMGTD_CUDA(ctx, cudaMemcpyAsync(rc_d, sys->rc_loc, sizeof(double) * na, cudaMemcpyHostToDevice, ctx->stream));
  }
  if (sys->rho_core) {   // frozen core density: xc only
    ctx->rho_core = (double*)A(gsz);
    if (!ctx->rho_core) return set_error(ctx, RMGTD_ENOMEM, "core density");
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->rho_core, sys->rho_core, gsz, cudaMemcpyHostToDevice,
                                    ctx->stream));
  }
  int rc = launch_vion(ctx, pos_d, Z_d, rc_d, na);
  if (rc) return rc;
  k_ion_energy<<<1, 256, 0, ctx->stream>>>(na, pos_d, Z_d, rc_d, eion_d);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_ion_energy");
  RMGTD_CUDA(ctx, cudaMemcpyAsync(&ctx->obs_host[0], eion_d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->E_ion = ctx->obs_host[0];

  rc = build_projectors(ctx, sys);
  if (rc) return rc;
  rc = setup_multigrid(ctx);
  if (rc) return rc;

  if (opt->orthonormalize) {
    rc = orthonormalize(ctx);
    if (rc) return rc;
  }
  if (opt->ground_state_scf > 0) {   // the Kohn-Sham ground state replaces phi0
    rc = ground_state_scf(ctx);
    if (rc) return rc;
  }
  rc = gram(ctx, ctx->phi, ctx->phi, nullptr, 0, 1, ctx->h3, nullptr, ctx->Smat, nullptr, nullptr,
            1, nullptr);
  if (rc) return rc;

  // H_core = h^3 Phi^T (T + V_loc + V_ext + V_NL) Phi, symmetrised
  {
    double* hphi = (double*)A(gsz * N);
    if (!hphi) return set_error(ctx, RMGTD_ENOMEM, "H Phi scratch");
    rc = apply_h_dev(ctx, ctx->phi, hphi, N, RMGTD_F64, nullptr);
    if (rc) return rc;
    rc = gram(ctx, ctx->phi, hphi, nullptr, 0, 1, ctx->h3, nullptr, ctx->H1, nullptr, nullptr, 0,
              nullptr);
    if (rc) return rc;
    k_symmetrize<<<std::max(1, (int)std::min<long>(ceil_div(NN, 256), 1024)), 256, 0, ctx->stream>>>(
        N, ctx->H1, ctx->Hcore);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_symmetrize");
    RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, hphi);
  }
  // M_q = h^3 Phi^T q Phi
  {
    double* q = (double*)A(3 * gsz);
    if (!q) return set_error(ctx, RMGTD_ENOMEM, "coordinate scratch");
    k_coords<<<std::max(1, (int)std::min<long>(ceil_div(Ng, 256), 4096)), 256, 0, ctx->stream>>>(
        ctx->nx, ctx->ny, ctx->nz, ctx->h, q);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_coords");
    for (int d = 0; d < 3; ++d) {
      rc = gram(ctx, ctx->phi, ctx->phi, q + d * Ng, 0, 1, ctx->h3, nullptr, ctx->M + d * NN,
                nullptr, nullptr, 1, nullptr);
      if (rc) return rc;
    }
    RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, q);
  }
  // P_0 = diag(f), H_0 = H[rho(P_0)], H_-1 = H_0
  k_diag_init<<<std::max(1, (int)std::min<long>(ceil_div(NN * nrep, 256), 1024)), 256, 0, ctx->stream>>>(
      N, nrep, ctx->f_dev, ctx->S0, ctx->A0);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_diag_init");
  if (opt->nonorthogonal) {   // S^-1 and P_0 = L^-T diag(f) L^-1 (replaces diag(f))
    rc = nonorth_setup(ctx);
    if (rc) return rc;
  }
  k_set_active<<<1, 32, 0, ctx->stream>>>(ctx->ctl, nrep, 1);
  ++ctx->launches;
  rc = dft_eval(ctx, ctx->S0, ctx->ctl, nullptr);
  if (rc) return rc;
  if (opt->subspace_scf > 0) {
    // SCF inside the orbital block: P <- mix(P, aufbau(H[rho(P)])) until stationary
    double* err_d = (double*)A(sizeof(double) * nrep);
    if (!err_d) return set_error(ctx, RMGTD_ENOMEM, "subspace SCF");
    std::vector<double> err_h(nrep);
    for (int it = 0; it < opt->subspace_scf; ++it) {
      rc = subspace_update(ctx, opt->subspace_mix, err_d);
      if (rc) return rc;
      rc = dft_eval(ctx, ctx->S0, ctx->ctl, nullptr);
      if (rc) return rc;
      RMGTD_CUDA(ctx, cudaMemcpyAsync(err_h.data(), err_d, sizeof(double) * nrep,
                                      cudaMemcpyDeviceToHost, ctx->stream));
      RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      ctx->subspace_iters = it + 1;
      ctx->subspace_err = *std::max_element(err_h.begin(), err_h.end());
      if (ctx->subspace_err <= opt->subspace_tol) break;
    }
  }
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->H0, ctx->H1, msz * nrep, cudaMemcpyDeviceToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Hm1, ctx->H1, msz * nrep, cudaMemcpyDeviceToDevice, ctx->stream));
  if (ctx->Hm2)
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Hm2, ctx->H1, msz * nrep, cudaMemcpyDeviceToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->S1, ctx->S0, msz * nrep, cudaMemcpyDeviceToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->A1, ctx->A0, msz * nrep, cudaMemcpyDeviceToDevice, ctx->stream));
  k_set_active<<<1, 32, 0, ctx->stream>>>(ctx->ctl, nrep, 0);
  ++ctx->launches;
  if (opt->grid_basis) {   // the occupied orbitals themselves are the propagated state
    rc = gridprop_setup(ctx);
    if (rc) return rc;
  }
  if (opt->precision == RMGTD_PREC_MIXED && !opt->grid_basis) {
    // reference state of the mixed path: the float64 set-up state (all replicas start in it)
    const size_t fsz = sizeof(float) * Ng;
    ctx->phi32 = (float*)A(fsz * N);
    // bfloat16 planes for the orbital-tiled tensor-core contractions (32 < N <= 256)
    rc = planes_setup(ctx);
    if (rc) return rc;
    // else the 32-point tiled copy, padded to whole 128-point tiles (the N <= 32 density kernel
    // loads 16 KB per tile; the tiled Gram kernel reads 32 x 32 boxes)
    if (!ctx->phi_pl) {
      const size_t phit_bytes = sizeof(float) * 32 * ((N + 31) / 32) * 128 * ((Ng + 127) / 128);
      ctx->phi32t = (float*)A(phit_bytes);
      if (!ctx->phi32t) return set_error(ctx, RMGTD_ENOMEM, "tiled orbitals");
      RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->phi32t, 0, phit_bytes, ctx->stream));
    }
    ctx->Sref = (double*)A(msz);
    ctx->Href = (double*)A(msz);
    ctx->rho_ref = (double*)A(gsz);
    ctx->vref = (double*)A(gsz);
    ctx->vh_ref = (double*)A(gsz);
    ctx->dv32 = (float*)A(fsz * nrep);
    ctx->dvh32 = (float*)A(fsz * nrep);
    ctx->dvh_prev32 = (float*)A(fsz * nrep);
    ctx->dvh_prev2_32 = (float*)A(fsz * nrep);
    {
      const long Np = ((N + 31) / 32) * 32;
      ctx->shat32 = (float*)A(sizeof(float) * Np * Np * nrep);
      if (ctx->shat32)
        RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->shat32, 0, sizeof(float) * Np * Np * nrep, ctx->stream));
    }
    ctx->pcg32_r = (float*)A(fsz * nrep);
    ctx->pcg32_z = (float*)A(fsz * nrep);
    ctx->pcg32_p = (float*)A(fsz * nrep);
    ctx->pcg32_Ap = (float*)A(fsz * nrep);
    ctx->pcg32_Az = (float*)A(fsz * nrep);
    ctx->drho32 = (float*)A(fsz * nrep);
    ctx->rho_ref32 = (float*)A(fsz);
    ctx->rho_mom_cap = 4L * nrep * std::max(1, ctx->num_sms);
    ctx->rho_mom = (double*)A(sizeof(double) * ctx->rho_mom_cap);
    ctx->ghost32 = (float*)A(fsz * 4);
    if (!ctx->phi32 || !ctx->pcg32_Az || !ctx->dvh32 || !ctx->Href || !ctx->vh_ref ||
        !ctx->drho32 || !ctx->ghost32 || !ctx->rho_ref32)
      return set_error(ctx, RMGTD_ENOMEM, "mixed-precision buffers");
    rc = to_float(ctx, ctx->phi, ctx->phi32, (long)N * Ng);
    if (rc) return rc;
    if (ctx->phi32t) {
      rc = tile_orbitals(ctx);
      if (rc) return rc;
    }
    rc = to_float(ctx, ctx->ghost, ctx->ghost32, 4L * Ng);
    if (rc) return rc;
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Sref, ctx->S0, msz, cudaMemcpyDeviceToDevice, ctx->stream));
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Href, ctx->H0, msz, cudaMemcpyDeviceToDevice, ctx->stream));
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->rho_ref, ctx->rho, gsz, cudaMemcpyDeviceToDevice, ctx->stream));
    // base of the xc increment: rho_ref, plus the frozen core when there is one
    ctx->rho_xc_ref = ctx->rho_ref;
    if (ctx->rho_core) {
      ctx->rho_xc_ref = (double*)A(gsz);
      if (!ctx->rho_xc_ref) return set_error(ctx, RMGTD_ENOMEM, "xc reference density");
      rc = add_fields(ctx, ctx->rho_ref, ctx->rho_core, ctx->rho_xc_ref, Ng);
      if (rc) return rc;
    }
    rc = to_float(ctx, ctx->rho_xc_ref, ctx->rho_ref32, Ng);
    if (rc) return rc;
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->vh_ref, ctx->vh, gsz, cudaMemcpyDeviceToDevice, ctx->stream));
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->vref, ctx->vhxc, gsz, cudaMemcpyDeviceToDevice, ctx->stream));
    RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->dvh32, 0, fsz * nrep, ctx->stream));
    RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->dv32, 0, fsz * nrep, ctx->stream));
    rc = planes_anchor_reset(ctx);
    if (rc) return rc;
    ctx->mixed = 1;
  }
  rc = hartree_reset_history(ctx);
  if (rc) return rc;
  return check_status(ctx, "create");
}

int rmgtd_create(const rmgtd_system* sys, const rmgtd_options* opt_in, rmgtd_ctx** out) {
  if (!out) return set_error(nullptr, RMGTD_EINVAL, "out is NULL");
  *out = nullptr;
  rmgtd_options opt;
  if (opt_in)
    opt = *opt_in;
  else
    rmgtd_default_options(&opt);
  if (!sys || !sys->phi0) return set_error(nullptr, RMGTD_EINVAL, "system or phi0 is NULL");
  if (sys->nx < 8 || sys->ny < 8 || sys->nz < 8 || !(sys->h > 0))
    return set_error(nullptr, RMGTD_EINVAL, "grid must be at least 8^3 with h > 0");
  if (sys->nocc < 1 || sys->nvirt < 0 || sys->nocc + sys->nvirt > 8192)
    return set_error(nullptr, RMGTD_EINVAL, "active space must have 1 <= N <= 8192");
  if (sys->natoms < 0 || (sys->natoms > 0 && (!sys->pos || !sys->Z || !sys->rc_loc)))
    return set_error(nullptr, RMGTD_EINVAL, "atom arrays missing");
  if (sys->nproj < 0 ||
      (sys->nproj > 0 && (!sys->proj_atom || !sys->proj_l || !sys->proj_rc || !sys->E_kb)))
    return set_error(nullptr, RMGTD_EINVAL, "projector arrays missing");
  if (opt.nrep < 1 || opt.nrep > 32) return set_error(nullptr, RMGTD_EINVAL, "nrep must be 1..32");
  if ((long long)sys->nx * sys->ny * sys->nz * opt.nrep >= (1ll << 31) - (1ll << 22))
    return set_error(nullptr, RMGTD_EINVAL, "nx * ny * nz * nrep must be below 2^31 - 2^22");
  if (!(opt.dt > 0) || !(opt.H_thrs > 0) || !(opt.dP_thrs > 0) || opt.max_scf < 1 ||
      opt.max_terms < 1 || !(opt.poisson_tol > 0) || opt.poisson_max_iter < 1)
    return set_error(nullptr, RMGTD_EINVAL, "invalid options");
  if (opt.precision != RMGTD_PREC_FP64 && opt.precision != RMGTD_PREC_MIXED)
    return set_error(nullptr, RMGTD_EINVAL, "unknown precision");
  if (opt.magnus_order == 0) opt.magnus_order = 1;
  if (opt.seed_order == 0) opt.seed_order = 1;
  if (opt.sm_budget < 0) return set_error(nullptr, RMGTD_EINVAL, "sm_budget must be >= 0");
  if (opt.seed_order != 1 && opt.seed_order != 2)
    return set_error(nullptr, RMGTD_EINVAL, "seed_order must be 1 or 2");
  if (opt.magnus_order != 1 && opt.magnus_order != 2)
    return set_error(nullptr, RMGTD_EINVAL, "magnus_order must be 1 or 2");
  if (opt.nonorthogonal && (opt.orthonormalize || opt.subspace_scf > 0 || opt.magnus_order != 1))
    return set_error(nullptr, RMGTD_EINVAL,
                     "nonorthogonal needs orthonormalize = 0, subspace_scf = 0 and magnus_order 1");
  if (opt.ground_state_scf < 0 || (opt.ground_state_scf > 0 && (!opt.orthonormalize || opt.nonorthogonal)))
    return set_error(nullptr, RMGTD_EINVAL, "ground_state_scf needs orthonormalize = 1 and nonorthogonal 0");
  if (opt.grid_basis &&
      (sys->nvirt != 0 || opt.magnus_order != 1 || opt.nonorthogonal || opt.subspace_scf > 0))
    return set_error(nullptr, RMGTD_EINVAL,
                     "grid_basis needs nvirt = 0, magnus_order 1, nonorthogonal 0 and subspace_scf 0");
  rmgtd_ctx* ctx = new rmgtd_ctx();
  int rc = create_impl(sys, &opt, ctx);
  if (rc != RMGTD_OK) {
    g_last_error = ctx->err;
    rmgtd_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return RMGTD_OK;
}

int rmgtd_apply_h(rmgtd_ctx* ctx, const void* x, void* hx, int ncols, int dtype, int rep) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (!x || !hx || ncols < 1 || rep < -1 || rep >= ctx->nrep)
    return set_error(ctx, RMGTD_EINVAL, "apply_h: bad arguments");
  if (rep >= 0) {
    const int rc = mixed_fields64(ctx);
    if (rc) return rc;
  }
  const double* vextra = (rep >= 0) ? ctx->vhxc + (long)rep * ctx->Ng : nullptr;
  return apply_h_dev(ctx, x, hx, ncols, dtype, vextra);
}

int rmgtd_kick(rmgtd_ctx* ctx, int rep, int axis, double kappa) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (rep < 0 || rep >= ctx->nrep || axis < 0 || axis > 2)
    return set_error(ctx, RMGTD_EINVAL, "kick: bad replica or axis");
  if (ctx->opt.grid_basis) return gridprop_kick(ctx, rep, axis, kappa);
  const long NN = (long)ctx->N * ctx->N;
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  const double* Mq = ctx->M + axis * NN;
  int rc = RMGTD_OK;
  if (ctx->opt.nonorthogonal) {   // Omega = -i kappa S^-1 M_q
    rc = nonorth_kick_matrix(ctx, axis);
    if (rc) return rc;
    Mq = ctx->Gm;
  }
  rc = eldyn(ctx, Mq, Mq, 0, kappa, ctx->S0 + rep * NN, ctx->A0 + rep * NN,
             ctx->S1 + rep * NN, ctx->A1 + rep * NN, nullptr, nullptr, rep, 1);
  if (rc) return rc;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->S0 + rep * NN, ctx->S1 + rep * NN, sizeof(double) * NN,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->A0 + rep * NN, ctx->A1 + rep * NN, sizeof(double) * NN,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  rc = refresh_fields(ctx);
  if (rc) return rc;
  return check_status(ctx, "kick");
}

// One SCF pass of Algorithm 1 (series, density, fields, H update) for every active replica.
static int enqueue_pass(rmgtd_ctx* ctx, cudaGraphConditionalHandle cond, int use_cond) {
  ph_begin(ctx, PH_ELDYN);
  // Omega's matrices: Hbar (+ the field), or S^-1 (Hbar + V) in a non-orthogonal basis, and
  // the Omega_2 term
  const double *Ha, *Hb, *febar, *D;
  long hstride;
  int rc = magnus_prepare(ctx, &Ha, &Hb, &hstride, &febar, &D);
  if (!rc)
    rc = eldyn(ctx, Ha, Hb, hstride, ctx->opt.dt, ctx->S0, ctx->A0, ctx->S1, ctx->A1, ctx->ctl,
               ctx->ctl, 0, ctx->nrep, ctx->mixed ? ctx->shat32 : nullptr, febar, D,
               ctx->mixed != 0);
  ph_end(ctx);
  if (rc) return rc;
  rc = dft_eval(ctx, ctx->S1, ctx->ctl, ctx->errbits);
  if (rc) return rc;
  ph_begin(ctx, PH_OTHER);
  rc = scf_control(ctx, ctx->errbits, cond, use_cond);
  ph_end(ctx);
  return rc;
}

// Capture one whole time step as a graph: H_1 extrapolation, a device-side while loop of
// SCF passes (each containing the Hartree CG while loop), then the shift.
// Record one time step of `ctx` into the capture active on `main` (ctx->stream is switched
// to it meanwhile): extrapolation [and the learned seed], a device-side while loop of SCF
// passes whose body is captured on ctx->aux[0], the shift [and the density history].
static int capture_step(rmgtd_ctx* ctx, cudaStream_t main) {
  for (int i = 0; i < 3; ++i)
    if (!ctx->aux[i]) RMGTD_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux[i], cudaStreamNonBlocking));
  cudaStream_t user = ctx->stream;
  ctx->stream = main;
  ctx->capturing = 1;
  const long long saved_launches = ctx->launches;
  // H_1 extrapolation, control reset and the Hartree guess in one launch; the learned seed
  // (which changes H_1 only) after it
  int rc = step_begin_extrapolate(ctx);
  if (!rc) rc = field_begin(ctx);
  if (!rc && ctx->net) rc = net_predict(ctx);
  cudaGraphConditionalHandle hs = 0;
  cudaGraph_t body = nullptr;
  if (!rc) rc = new_handle(ctx, &hs, true);
  if (!rc) rc = add_while(ctx, hs, &body);
  if (!rc) {
    cudaError_t e = cudaStreamBeginCaptureToGraph(ctx->aux[0], body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      rc = cuda_check(ctx, e, "cudaStreamBeginCaptureToGraph");
    } else {
      ctx->stream = ctx->aux[0];
      const long long l0 = ctx->launches;
      rc = enqueue_pass(ctx, hs, 1);
      ctx->cap_scf = (int)(ctx->launches - l0);
      ctx->stream = main;
      cudaGraph_t out;
      e = cudaStreamEndCapture(ctx->aux[0], &out);
      if (!rc && e != cudaSuccess) rc = cuda_check(ctx, e, "end of SCF body capture");
    }
  }
  if (!rc) rc = step_end(ctx);
  if (!rc && ctx->net) rc = net_history_shift(ctx);
  // kernels of the top level: everything captured outside the SCF body
  ctx->cap_top = (int)(ctx->launches - saved_launches) - ctx->cap_scf;
  ctx->launches = saved_launches;
  ctx->capturing = 0;
  ctx->stream = user;
  return rc;
}

// Capture one whole time step as a graph (on a library-owned stream: the caller's stream
// may be the legacy default stream, which cannot be captured); launched on the caller's.
static int build_step_graph(rmgtd_ctx* ctx) {
  for (int i = 0; i < 3; ++i)
    if (!ctx->aux[i]) RMGTD_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux[i], cudaStreamNonBlocking));
  cudaStream_t main = ctx->aux[2];
  RMGTD_CUDA(ctx, cudaStreamBeginCapture(main, cudaStreamCaptureModeRelaxed));
  const int rc = capture_step(ctx, main);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(main, &g);
  if (rc) return rc;   // a part-way capture is not destroyed (see rmgtd_batch_create)
  RMGTD_CUDA(ctx, e);
  ctx->step_graph = g;
  RMGTD_CUDA(ctx, cudaGraphInstantiate(&ctx->step_exec, g, 0));
  return RMGTD_OK;
}

// Eager step: the host reads the control blocks after every pass.
static int eager_step(rmgtd_ctx* ctx) {
  // H_1 extrapolation, control reset and the Hartree guess in one launch; the learned seed
  // (which changes H_1 only) after it
  int rc = step_begin_extrapolate(ctx);
  if (!rc) rc = field_begin(ctx);
  if (!rc && ctx->net) rc = net_predict(ctx);
  if (rc) return rc;
  for (int pass = 0; pass < ctx->opt.max_scf; ++pass) {
    rc = enqueue_pass(ctx, 0, 0);
    if (rc) return rc;
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->ctl_host, ctx->ctl, sizeof(RepCtl) * ctx->nrep,
                                    cudaMemcpyDeviceToHost, ctx->stream));
    RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    bool any = false;
    for (int r = 0; r < ctx->nrep; ++r) any |= ctx->ctl_host[r].active != 0;
    if (!any) break;
  }
  ph_begin(ctx, PH_OTHER);
  rc = step_end(ctx);
  if (!rc && ctx->net) rc = net_history_shift(ctx);
  ph_end(ctx);
  return rc;
}

// After a chunk of `chunk` launched steps: copy the per-step statistics out (to
// stats[done_total ..] when given), advance time and step count, report a failed step.
// After a failed step the kept state (P_0, H_0, H_-1 of the last completed step) is intact,
// but the grid fields and the Hartree guess history hold the failed step's values (non-finite
// after a divergence): rebuild them from P_0, the Hartree solve starting from zero.  The
// failed step's error message is kept.
static void recover_after_failed_step(rmgtd_ctx* ctx) {
  const std::string msg = ctx->err;
  if (cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream) == cudaSuccess &&
      cudaMemsetAsync(ctx->vh, 0, sizeof(double) * ctx->Ng * ctx->nrep, ctx->stream) ==
          cudaSuccess &&
      refresh_fields(ctx) == RMGTD_OK)
    cudaStreamSynchronize(ctx->stream);
  ctx->err = msg;
}

static int finish_chunk(rmgtd_ctx* ctx, int chunk, int done_total, rmgtd_stats* stats, int* done_out) {
  const int nrep = ctx->nrep;
  int* hdr = (int*)&ctx->ctl_host[nrep];  // scratch: done, failed, status
  RMGTD_CUDA(ctx, cudaMemcpyAsync(&hdr[0], ctx->done_steps, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(&hdr[1], ctx->failed, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(&hdr[2], ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->stats_host, ctx->stats_dev, sizeof(RepCtl) * chunk * nrep,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const int done = hdr[0], failed = hdr[1], gstatus = hdr[2];
  const int recorded = std::min(chunk, done + (failed ? 1 : 0));
  int worst = RMGTD_OK;
  for (int k = 0; k < recorded; ++k) {
    for (int r = 0; r < nrep; ++r) {
      const RepCtl& c = ctx->stats_host[(long)k * nrep + r];
      if (stats) {
        rmgtd_stats& o = stats[(long)(done_total + k) * nrep + r];
        o.passes = c.passes;
        o.terms_max = c.terms_max;
        o.terms_sum = c.terms_sum;
        o.status = c.status;
        o.H_err = c.H_err;
      }
      if (k == done && c.status != 0 && worst == RMGTD_OK) worst = c.status;
    }
  }
  ctx->steps += done;
  ctx->t += done * ctx->opt.dt;
  *done_out = done;
  if (failed) {
    if (worst == RMGTD_OK) worst = gstatus ? gstatus : RMGTD_ENOTCONVERGED;
    char buf[128];
    snprintf(buf, sizeof(buf), "step %lld failed with status %d", ctx->steps + 1, worst);
    ph_flush(ctx);
    const int rc = set_error(ctx, worst, buf);
    recover_after_failed_step(ctx);
    return rc;
  }
  return RMGTD_OK;
}

int rmgtd_step(rmgtd_ctx* ctx, int nsteps, rmgtd_stats* stats) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (nsteps < 0) return set_error(ctx, RMGTD_EINVAL, "nsteps < 0");
  if (ctx->in_batch) return set_error(ctx, RMGTD_ESTATE, "context belongs to a batch: step the batch");
  if (ctx->opt.grid_basis) {   // host-driven steps of the orbitals on the grid
    for (int i = 0; i < nsteps; ++i) {
      const int rc = gridprop_step(ctx, stats ? stats + (long)i * ctx->nrep : nullptr);
      if (rc) return rc;
    }
    return ph_flush(ctx);
  }
  if (ctx->opt.use_graph && !ctx->step_exec) {
    int rc = build_step_graph(ctx);
    if (rc) return rc;
  }
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->failed, 0, sizeof(int), ctx->stream));
  if (ctx->mixed && nsteps > 0) ctx->fields_stale = 1;
  int done_total = 0;
  while (done_total < nsteps) {
    const int chunk = std::min(nsteps - done_total, ctx->stats_cap);
    RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->done_steps, 0, sizeof(int), ctx->stream));
    for (int i = 0; i < chunk; ++i) {
      if (ctx->step_exec) {
        RMGTD_CUDA(ctx, cudaGraphLaunch(ctx->step_exec, ctx->stream));
        ctx->graph_steps += 1;
      } else {
        int rc = eager_step(ctx);
        if (rc) return rc;
      }
    }
    int done = 0;
    int rc = finish_chunk(ctx, chunk, done_total, stats, &done);
    if (rc) return rc;
    done_total += done;
  }
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return ph_flush(ctx);
}

// ---- autotuner: time the launch alternatives on this context's shapes ----------------------
// Each candidate runs on scratch outputs (state untouched): 2 warm-up and 5 timed calls with
// CUDA events on the context's stream; the smallest median wins.  The Hartree candidates
// solve from a zero initial guess into a scratch unknown.
int rmgtd_autotune(rmgtd_ctx* ctx, int choice[4]) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (ctx->in_batch) return set_error(ctx, RMGTD_ESTATE, "autotune: context belongs to a batch");
  if (ctx->opt.grid_basis) return set_error(ctx, RMGTD_ESTATE, "autotune: grid-basis context");
  const int nrep = ctx->nrep;
  const long Ng = ctx->Ng, NN = (long)ctx->N * ctx->N;
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double* rho_s = (double*)dev_alloc(ctx, sizeof(double) * Ng * nrep);
  float* drho_s = (float*)dev_alloc(ctx, sizeof(float) * Ng * nrep);
  double* gram_s = (double*)dev_alloc(ctx, sizeof(double) * NN * nrep);
  void* x_s = dev_alloc(ctx, sizeof(double) * Ng * nrep);
  if (!rho_s || !drho_s || !gram_s || !x_s) return set_error(ctx, RMGTD_ENOMEM, "autotune scratch");
  cudaEvent_t e0, e1;
  RMGTD_CUDA(ctx, cudaEventCreate(&e0));
  RMGTD_CUDA(ctx, cudaEventCreate(&e1));
  int rc = RMGTD_OK;
  // median of 5 timed calls of `fn` (after 2 untimed); `prep` runs before each call, untimed
  auto timed = [&](auto fn, auto prep, float* ms) -> int {
    float t[5];
    for (int it = 0; it < 7; ++it) {
      int r = prep();
      if (r) return r;
      RMGTD_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
      r = fn();
      if (r) return r;
      RMGTD_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
      RMGTD_CUDA(ctx, cudaEventSynchronize(e1));
      if (it >= 2) RMGTD_CUDA(ctx, cudaEventElapsedTime(&t[it - 2], e0, e1));
    }
    std::sort(t, t + 5);
    *ms = t[2];
    return RMGTD_OK;
  };
  auto none = [&]() { return RMGTD_OK; };
  const int launches0 = (int)ctx->launches;
  if (ctx->mixed) {
    // density: CTAs per SM of the tensor-core kernel (also leaves valid Shat / drho inputs)
    rc = rho_dev_mixed(ctx, ctx->S0, rho_s, nullptr, nrep);
    const int keep_rho = ctx->tune_rho_blocks;
    float best = 1e30f;
    int best_b = keep_rho;
    for (int b : {1, 2, 3, 4}) {
      if (rc) break;
      ctx->tune_rho_blocks = b;
      float ms;
      int r = timed([&]() { return rho_tc(ctx, rho_s, drho_s, nullptr, nrep); }, none, &ms);
      if (r > 0) break;   // shape outside the tensor-core kernel
      if (r < 0) {
        rc = r;
        break;
      }
      if (ms < best) best = ms, best_b = b;
    }
    ctx->tune_rho_blocks = best_b;
    // Gram: kernel x CTAs per SM
    best = 1e30f;
    int best_tc = ctx->tune_gram_tc, best_gb = ctx->tune_gram_blocks;
    for (int tcv : {0, 1})
      for (int b : {1, 2, 4, 8}) {
        if (rc) break;
        ctx->tune_gram_tc = tcv;
        ctx->tune_gram_blocks = b;
        float ms;
        rc = timed([&]() { return gram_mixed(ctx, ctx->dv32, Ng, nrep, ctx->h3, ctx->Href, gram_s,
                                             nullptr, nullptr); }, none, &ms);
        if (!rc && ms < best) best = ms, best_tc = tcv, best_gb = b;
      }
    ctx->tune_gram_tc = best_tc;
    ctx->tune_gram_blocks = best_gb;
  }
  // Hartree: blocks of the persistent solve (SMs / div), from a zero guess
  {
    float best = 1e30f;
    int best_d = ctx->tune_coop_div;
    ctx->tune_x = x_s;
    const size_t xb = (ctx->mixed ? sizeof(float) : sizeof(double)) * Ng * nrep;
    for (int d : {1, 2, 4}) {
      if (rc) break;
      ctx->tune_coop_div = d;
      float ms;
      rc = timed([&]() { return hartree_coop(ctx, ctx->rho, ctx->vh, nullptr, 0, nrep, ctx->mixed); },
                 [&]() {
                   const cudaError_t me = cudaMemsetAsync(x_s, 0, xb, ctx->stream);
                   return me == cudaSuccess ? (int)RMGTD_OK : cuda_check(ctx, me, "memset");
                 },
                 &ms);
      if (!rc && ms < best) best = ms, best_d = d;
    }
    ctx->tune_x = nullptr;
    ctx->tune_coop_div = best_d;
  }
  ctx->launches = launches0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the candidates may have flagged their scratch solves; the state is untouched
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  dev_free(ctx, rho_s);
  dev_free(ctx, drho_s);
  dev_free(ctx, gram_s);
  dev_free(ctx, x_s);
  if (rc) return rc;
  // launch configurations are baked into the step graph: rebuild it
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
  ctx->step_exec = nullptr;
  ctx->step_graph = nullptr;
  if (choice) {
    choice[0] = ctx->tune_rho_blocks;
    choice[1] = ctx->tune_gram_tc;
    choice[2] = ctx->tune_gram_blocks;
    choice[3] = ctx->tune_coop_div;
  }
  return RMGTD_OK;
}

int rmgtd_set_tuning(rmgtd_ctx* ctx, const int choice[4]) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (!choice) return set_error(ctx, RMGTD_EINVAL, "set_tuning: choice is NULL");
  if (ctx->in_batch) return set_error(ctx, RMGTD_ESTATE, "set_tuning: context belongs to a batch");
  const auto one_of = [](int v, std::initializer_list<int> s) {
    for (int x : s)
      if (v == x) return true;
    return false;
  };
  if (choice[0] < 1 || choice[0] > 4 || !one_of(choice[1], {0, 1}) ||
      !one_of(choice[2], {1, 2, 4, 8}) || !one_of(choice[3], {1, 2, 4}))
    return set_error(ctx, RMGTD_EINVAL, "set_tuning: value out of range");
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->tune_rho_blocks = choice[0];
  ctx->tune_gram_tc = choice[1];
  ctx->tune_gram_blocks = choice[2];
  ctx->tune_coop_div = choice[3];
  // launch configurations are baked into the step graph: rebuild it
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
  ctx->step_exec = nullptr;
  ctx->step_graph = nullptr;
  return RMGTD_OK;
}

int rmgtd_set_hartree_preconditioner(rmgtd_ctx* ctx, int kind) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (kind != RMGTD_PRECOND_DST && kind != RMGTD_PRECOND_MG)
    return set_error(ctx, RMGTD_EINVAL, "set_hartree_preconditioner: unknown kind");
  if (ctx->in_batch)
    return set_error(ctx, RMGTD_ESTATE, "set_hartree_preconditioner: context belongs to a batch");
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->hartree_precond = kind;
  // the solve's arguments are baked into the step graph: rebuild it
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
  ctx->step_exec = nullptr;
  ctx->step_graph = nullptr;
  return RMGTD_OK;
}

int rmgtd_get_tuning(const rmgtd_ctx* ctx, int choice[4]) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (!choice) return RMGTD_EINVAL;
  choice[0] = ctx->tune_rho_blocks;
  choice[1] = ctx->tune_gram_tc;
  choice[2] = ctx->tune_gram_blocks;
  choice[3] = ctx->tune_coop_div;
  return RMGTD_OK;
}

// ---- several systems in one graph per step (batched launch of independent systems) ---------
struct rmgtd_batch {
  std::vector<rmgtd_ctx*> ctxs;
  cudaStream_t stream = nullptr;     // the contexts' common stream (launch stream)
  cudaStream_t capture = nullptr;    // library-owned capture stream
  std::vector<cudaStream_t> branch;  // one forked capture stream per context (concurrent)
  std::vector<cudaEvent_t> events;   // fork and join events of the capture
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void batch_release(rmgtd_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->branch)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->events)
    if (e) cudaEventDestroy(e);
  if (b->capture) cudaStreamDestroy(b->capture);
  delete b;
}

int rmgtd_batch_create(rmgtd_ctx* const* ctxs, int n, rmgtd_batch** out) {
  if (!out) return set_error(nullptr, RMGTD_EINVAL, "batch_create: out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1) return set_error(nullptr, RMGTD_EINVAL, "batch_create: no contexts");
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return set_error(nullptr, RMGTD_EINVAL, "batch_create: NULL context");
    if (ctxs[i]->in_batch) return set_error(nullptr, RMGTD_EINVAL, "batch_create: context already in a batch");
    if (ctxs[i]->opt.grid_basis) return set_error(nullptr, RMGTD_ESTATE, "batch_create: grid-basis context");
    if (ctxs[i]->stream != ctxs[0]->stream)
      return set_error(nullptr, RMGTD_EINVAL, "batch_create: contexts must share one stream");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return set_error(nullptr, RMGTD_EINVAL, "batch_create: context repeated");
  }
  rmgtd_batch* b = new rmgtd_batch();
  b->ctxs.assign(ctxs, ctxs + n);
  b->stream = ctxs[0]->stream;
  auto fail = [&](int code, const std::string& msg) {
    batch_release(b);
    return set_error(nullptr, code, msg);
  };
  // contexts with an SM budget run concurrently: each one's step is captured on its own
  // stream forked from the capture stream and joined back; without budgets (every context
  // sized to the whole GPU) they run one after another on the capture stream
  bool concurrent = n > 1;
  for (auto* c : b->ctxs) concurrent = concurrent && c->opt.sm_budget > 0;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess)
    return fail(RMGTD_ECUDA, "batch_create: stream");
  if (concurrent) {
    b->branch.assign(n, nullptr);
    b->events.assign(n + 1, nullptr);
    for (int i = 0; i < n; ++i)
      if (cudaStreamCreateWithFlags(&b->branch[i], cudaStreamNonBlocking) != cudaSuccess)
        return fail(RMGTD_ECUDA, "batch_create: branch stream");
    for (int i = 0; i <= n; ++i)
      if (cudaEventCreateWithFlags(&b->events[i], cudaEventDisableTiming) != cudaSuccess)
        return fail(RMGTD_ECUDA, "batch_create: event");
  }
  if (cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return fail(RMGTD_ECUDA, "batch_create: begin capture");
  int rc = RMGTD_OK;
  int bad = -1;
  if (concurrent && cudaEventRecord(b->events[n], b->capture) != cudaSuccess) {
    rc = RMGTD_ECUDA;
    bad = 0;
  }
  for (int i = 0; i < n && !rc; ++i) {
    cudaStream_t s = b->capture;
    if (concurrent) {
      s = b->branch[i];
      if (cudaStreamWaitEvent(s, b->events[n], 0) != cudaSuccess) rc = RMGTD_ECUDA;
    }
    if (!rc) rc = capture_step(b->ctxs[i], s);
    if (!rc && concurrent &&
        (cudaEventRecord(b->events[i], s) != cudaSuccess ||
         cudaStreamWaitEvent(b->capture, b->events[i], 0) != cudaSuccess))
      rc = RMGTD_ECUDA;
    if (rc) bad = i;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->capture, &g);
  // a graph whose capture failed part-way (inside a conditional body) is left to the driver
  // rather than destroyed: it is never instantiated or launched
  if (rc) {
    b->graph = nullptr;
    return fail(rc, std::string("batch_create: context ") + std::to_string(bad) + ": " +
                        (b->ctxs[bad]->err.empty() ? "capture failed" : b->ctxs[bad]->err));
  }
  b->graph = g;
  if (e != cudaSuccess) return fail(RMGTD_ECUDA, std::string("batch_create: ") + cudaGetErrorString(e));
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess)
    return fail(RMGTD_ECUDA, "batch_create: graph instantiation");
  for (auto* c : b->ctxs) c->in_batch = 1;
  *out = b;
  return RMGTD_OK;
}

void rmgtd_batch_destroy(rmgtd_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto* c : b->ctxs) c->in_batch = 0;
  batch_release(b);
}

int rmgtd_batch_step(rmgtd_batch* b, int nsteps, rmgtd_stats* const* stats) {
  if (!b) return set_error(nullptr, RMGTD_EINVAL, "batch_step: NULL batch");
  if (nsteps < 0) return set_error(nullptr, RMGTD_EINVAL, "batch_step: nsteps < 0");
  int cap = b->ctxs[0]->stats_cap;
  for (auto* c : b->ctxs) {
    cap = std::min(cap, c->stats_cap);
    RMGTD_CUDA(c, cudaMemsetAsync(c->failed, 0, sizeof(int), b->stream));
    if (c->mixed && nsteps > 0) c->fields_stale = 1;
  }
  int done_total = 0;
  while (done_total < nsteps) {
    const int chunk = std::min(nsteps - done_total, cap);
    for (auto* c : b->ctxs) RMGTD_CUDA(c, cudaMemsetAsync(c->done_steps, 0, sizeof(int), b->stream));
    for (int i = 0; i < chunk; ++i) {
      const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
      if (e != cudaSuccess) return set_error(nullptr, RMGTD_ECUDA, cudaGetErrorString(e));
    }
    int done_min = chunk, first_err = RMGTD_OK;
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
      rmgtd_ctx* c = b->ctxs[i];
      c->graph_steps += chunk;
      int done = 0;
      const int rc = finish_chunk(c, chunk, done_total, stats ? stats[i] : nullptr, &done);
      if (rc && first_err == RMGTD_OK) {
        first_err = rc;
        set_error(nullptr, rc, std::string("batch_step: context ") + std::to_string(i) + ": " + c->err);
      }
      done_min = std::min(done_min, done);
    }
    if (first_err) return first_err;
    done_total += done_min;
  }
  return RMGTD_OK;
}


int rmgtd_profile(rmgtd_ctx* ctx, int enable) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  int rc = ph_flush(ctx);
  if (rc) return rc;
  if (enable && ctx->ev_pool.empty()) {
    ctx->ev_pool.resize(2 * kEvPairs);
    ctx->ev_phase.resize(kEvPairs);
    for (auto& e : ctx->ev_pool) RMGTD_CUDA(ctx, cudaEventCreate(&e));
  }
  ctx->profile = enable ? 1 : 0;
  for (int i = 0; i < 8; ++i) {
    ctx->phase_ms[i] = 0;
    ctx->phase_calls[i] = 0;
  }
  ctx->launches = 0;
  ctx->graph_steps = 0;
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->kexec, 0, 4 * sizeof(unsigned long long), ctx->stream));
  return RMGTD_OK;
}

int rmgtd_profile_read(rmgtd_ctx* ctx, double* phase_ms, long long* phase_calls,
                       long long* launches) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  int rc = ph_flush(ctx);
  if (rc) return rc;
  for (int i = 0; i < RMGTD_NPHASES; ++i) {
    if (phase_ms) phase_ms[i] = ctx->phase_ms[i];
    if (phase_calls) phase_calls[i] = ctx->phase_calls[i];
  }
  if (launches) {
    unsigned long long kx[2] = {0, 0};
    RMGTD_CUDA(ctx, cudaMemcpy(kx, ctx->kexec, sizeof(kx), cudaMemcpyDeviceToHost));
    *launches = ctx->launches + ctx->graph_steps * ctx->cap_top + (long long)kx[0] * ctx->cap_scf;
  }
  return RMGTD_OK;
}

int rmgtd_profile_counters(rmgtd_ctx* ctx, long long* hartree_solves,
                           long long* hartree_iterations) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  unsigned long long kx[4] = {0, 0, 0, 0};
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpy(kx, ctx->kexec, sizeof(kx), cudaMemcpyDeviceToHost));
  if (hartree_solves) *hartree_solves = (long long)kx[2];
  if (hartree_iterations) *hartree_iterations = (long long)kx[3];
  return RMGTD_OK;
}

int rmgtd_surrogate_load(rmgtd_ctx* ctx, const char* path, rmgtd_net** net_out) {
  if (!ctx || !path || !net_out) return set_error(ctx, RMGTD_EINVAL, "surrogate_load: NULL argument");
  *net_out = nullptr;
  rmgtd_net* net = nullptr;
  int rc = rmgtd_net_create(ctx->nx, ctx->ny, ctx->nz, ctx->nrep, ctx->stream, &net);
  if (rc) return set_error(ctx, rc, std::string("surrogate_load: ") + rmgtd_last_error(nullptr));
  rc = rmgtd_net_load(net, path);
  if (!rc) rc = rmgtd_attach_net(ctx, net);
  if (rc) {
    const std::string msg = ctx->err.empty() ? rmgtd_last_error(nullptr) : ctx->err;
    rmgtd_net_destroy(net);
    return set_error(ctx, rc, "surrogate_load: " + msg);
  }
  *net_out = net;
  return RMGTD_OK;
}

int rmgtd_attach_net(rmgtd_ctx* ctx, rmgtd_net* net) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (ctx->in_batch) return set_error(ctx, RMGTD_ESTATE, "attach_net: context belongs to a batch");
  if (ctx->opt.grid_basis) return set_error(ctx, RMGTD_ESTATE, "attach_net: grid-basis context");
  if (net) {
    int nx, ny, nz;
    net_grid_points(net, &nx, &ny, &nz);
    if (nx != ctx->nx || ny != ctx->ny || nz != ctx->nz)
      return set_error(ctx, RMGTD_EINVAL, "attach_net: network grid differs from the context's");
    if (net_batch_cap(net) < ctx->nrep)
      return set_error(ctx, RMGTD_EINVAL, "attach_net: network max_batch < nrep");
    if (!ctx->rho_h1) {
      const size_t g = sizeof(double) * ctx->Ng * ctx->nrep, f = sizeof(float) * ctx->Ng * ctx->nrep;
      ctx->net_x = (float*)dev_alloc(ctx, 3 * f);
      ctx->net_y = (float*)dev_alloc(ctx, f);
      ctx->net_dv32 = (float*)dev_alloc(ctx, f);
      ctx->net_dv64 = (double*)dev_alloc(ctx, g);
      ctx->rho_h1 = (double*)dev_alloc(ctx, g);
      ctx->rho_h2 = (double*)dev_alloc(ctx, g);
      ctx->rho_start = (double*)dev_alloc(ctx, g);
      if (!ctx->net_x || !ctx->net_y || !ctx->net_dv32 || !ctx->net_dv64 || !ctx->rho_h1 ||
          !ctx->rho_h2 || !ctx->rho_start)
        return set_error(ctx, RMGTD_ENOMEM, "attach_net: predictor buffers");
    }
  }
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->net = net;
  // the step graph changes with the predictor: rebuild it on the next step
  if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
  if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
  ctx->step_exec = nullptr;
  ctx->step_graph = nullptr;
  if (net) {
    int rc = mixed_fields64(ctx);   // the history starts from the current float64 density
    if (rc) return rc;
    rc = net_history_reset(ctx);
    if (rc) return rc;
  }
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

int rmgtd_get_field(rmgtd_ctx* ctx, int which, int rep, double* dev_out) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (rep < 0 || rep >= ctx->nrep || !dev_out) return set_error(ctx, RMGTD_EINVAL, "get_field: bad arguments");
  const double* src = which == RMGTD_FIELD_RHO ? ctx->rho : which == RMGTD_FIELD_VHXC ? ctx->vhxc : nullptr;
  if (!src) return set_error(ctx, RMGTD_EINVAL, "get_field: unknown field");
  const int rc = mixed_fields64(ctx);
  if (rc) return rc;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(dev_out, src + (long)rep * ctx->Ng, sizeof(double) * ctx->Ng,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

int rmgtd_density(rmgtd_ctx* ctx, int rep, double* rho_host) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (rep < 0 || rep >= ctx->nrep || !rho_host) return set_error(ctx, RMGTD_EINVAL, "density: bad arguments");
  int rc = ctx->opt.grid_basis ? gridprop_observables(ctx)
                               : rho_dev(ctx, ctx->S0, ctx->rho, nullptr, ctx->nrep);
  if (rc) return rc;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(rho_host, ctx->rho + (long)rep * ctx->Ng, sizeof(double) * ctx->Ng,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

static int fetch_obs(rmgtd_ctx* ctx) {
  int rc = observables(ctx);
  if (rc) return rc;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->obs_host, ctx->obs, sizeof(double) * 8 * ctx->nrep,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

int rmgtd_dipole(rmgtd_ctx* ctx, int rep, double mu[3]) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (rep < 0 || rep >= ctx->nrep || !mu) return set_error(ctx, RMGTD_EINVAL, "dipole: bad arguments");
  if (ctx->opt.grid_basis) {
    const int rc = gridprop_observables(ctx);
    if (rc) return rc;
    gridprop_read(ctx, rep, mu, nullptr, nullptr);
    return RMGTD_OK;
  }
  int rc = fetch_obs(ctx);
  if (rc) return rc;
  for (int d = 0; d < 3; ++d) mu[d] = ctx->obs_host[8 * rep + d];
  return RMGTD_OK;
}

int rmgtd_energy(rmgtd_ctx* ctx, int rep, double* E) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (rep < 0 || rep >= ctx->nrep || !E) return set_error(ctx, RMGTD_EINVAL, "energy: bad arguments");
  if (ctx->opt.grid_basis) {
    const int rc = gridprop_observables(ctx);
    if (rc) return rc;
    gridprop_read(ctx, rep, nullptr, E, nullptr);
    return RMGTD_OK;
  }
  int rc = mixed_fields64(ctx);
  if (rc) return rc;
  rc = fetch_obs(ctx);
  if (rc) return rc;
  *E = ctx->obs_host[8 * rep + 4];
  return RMGTD_OK;
}

static double* matrix_ptr(rmgtd_ctx* ctx, int which, int rep, bool* shared) {
  const long NN = (long)ctx->N * ctx->N;
  *shared = false;
  switch (which) {
    case RMGTD_MAT_P_RE: return ctx->S0 + rep * NN;
    case RMGTD_MAT_P_IM: return ctx->A0 + rep * NN;
    case RMGTD_MAT_H0: return ctx->H0 + rep * NN;
    case RMGTD_MAT_HM1: return ctx->Hm1 + rep * NN;
  }
  *shared = true;
  switch (which) {
    case RMGTD_MAT_HCORE: return ctx->Hcore;
    case RMGTD_MAT_MX: return ctx->M;
    case RMGTD_MAT_MY: return ctx->M + NN;
    case RMGTD_MAT_MZ: return ctx->M + 2 * NN;
    case RMGTD_MAT_S: return ctx->Smat;
  }
  return nullptr;
}

int rmgtd_get_matrix(rmgtd_ctx* ctx, int which, int rep, double* host_out) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (ctx->opt.grid_basis) return set_error(ctx, RMGTD_ESTATE, "get_matrix: grid-basis context (no P)");
  if (rep < 0 || rep >= ctx->nrep || !host_out) return set_error(ctx, RMGTD_EINVAL, "get_matrix: bad arguments");
  bool shared;
  double* p = matrix_ptr(ctx, which, rep, &shared);
  if (!p) return set_error(ctx, RMGTD_EINVAL, "get_matrix: unknown matrix");
  RMGTD_CUDA(ctx, cudaMemcpyAsync(host_out, p, sizeof(double) * ctx->N * ctx->N,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

int rmgtd_set_matrix(rmgtd_ctx* ctx, int which, int rep, const double* host_in) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (ctx->opt.grid_basis) return set_error(ctx, RMGTD_ESTATE, "set_matrix: grid-basis context (no P)");
  if (rep < 0 || rep >= ctx->nrep || !host_in) return set_error(ctx, RMGTD_EINVAL, "set_matrix: bad arguments");
  bool shared;
  double* p = matrix_ptr(ctx, which, rep, &shared);
  if (!p || shared) return set_error(ctx, RMGTD_EINVAL, "set_matrix: only P, H0, H-1 are writable");
  RMGTD_CUDA(ctx, cudaMemcpyAsync(p, host_in, sizeof(double) * ctx->N * ctx->N,
                                  cudaMemcpyHostToDevice, ctx->stream));
  if (which == RMGTD_MAT_HM1 && ctx->Hm2)   // the quadratic seed restarts from H_-1
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Hm2 + (long)rep * ctx->N * ctx->N, p,
                                    sizeof(double) * ctx->N * ctx->N, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
  if (which == RMGTD_MAT_P_RE) {
    int rc = refresh_fields(ctx);
    if (rc) return rc;
  }
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

int rmgtd_hartree(rmgtd_ctx* ctx, const double* rho_dev, double* vh_dev) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (!rho_dev || !vh_dev) return set_error(ctx, RMGTD_EINVAL, "hartree: NULL pointer");
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  int rc = hartree_coop(ctx, rho_dev, vh_dev, nullptr, 0, 1, 0);
  if (rc) return rc;
  return check_status(ctx, "hartree");
}

int rmgtd_xc(rmgtd_ctx* ctx, const double* rho_dev, double* vxc_dev, double* exc_dev, size_t n) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (!rho_dev || !vxc_dev || n == 0) return set_error(ctx, RMGTD_EINVAL, "xc: bad arguments");
  int rc = launch_lda(ctx, rho_dev, nullptr, 0, vxc_dev, exc_dev, nullptr, nullptr, (long)n, nullptr,
                      1, (long)n, 1, false);
  if (rc) return rc;
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

int rmgtd_xc_increment(rmgtd_ctx* ctx, const double* rho0_dev, const float* drho_dev,
                       float* dvxc_dev, size_t n) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (!rho0_dev || !drho_dev || !dvxc_dev || n == 0)
    return set_error(ctx, RMGTD_EINVAL, "xc_increment: bad arguments");
  int rc = launch_xc_increment(ctx, rho0_dev, drho_dev, dvxc_dev, (long)n);
  if (rc) return rc;
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

int rmgtd_set_field(rmgtd_ctx* ctx, int rep, const double* E_xyz, int nsamp) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (rep < 0 || rep >= ctx->nrep || nsamp < 0 || (nsamp > 0 && !E_xyz))
    return set_error(ctx, RMGTD_EINVAL, "set_field: bad replica, count or NULL samples");
  if (ctx->in_batch) return set_error(ctx, RMGTD_ESTATE, "set_field: context belongs to a batch");
  for (int i = 0; i < 3 * nsamp; ++i)
    if (!std::isfinite(E_xyz[i])) return set_error(ctx, RMGTD_EINVAL, "set_field: non-finite sample");
  ctx->fld_host[rep].assign(E_xyz, E_xyz + 3 * (size_t)nsamp);
  int cap = 0, on = 0;
  for (const auto& v : ctx->fld_host) {
    cap = std::max(cap, (int)(v.size() / 3));
    on |= !v.empty();
  }
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  const bool regrow = cap > ctx->fld_cap;   // the captured kernels hold the old buffer and pitch
  if (regrow) {
    dev_free(ctx, ctx->fld_samples);
    ctx->fld_samples = (double*)dev_alloc(ctx, sizeof(double) * 3 * (size_t)cap * ctx->nrep);
    if (!ctx->fld_samples) {
      ctx->fld_cap = 0;
      ctx->fld_on = 0;
      return set_error(ctx, RMGTD_ENOMEM, "set_field: samples");
    }
    ctx->fld_cap = cap;
  }
  std::vector<int> ns(ctx->nrep);
  if (ctx->fld_cap > 0) {
    std::vector<double> all(3 * (size_t)ctx->fld_cap * ctx->nrep, 0.0);
    for (int r = 0; r < ctx->nrep; ++r) {
      std::copy(ctx->fld_host[r].begin(), ctx->fld_host[r].end(),
                all.begin() + 3 * (size_t)ctx->fld_cap * r);
      ns[r] = (int)(ctx->fld_host[r].size() / 3);
    }
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->fld_samples, all.data(), sizeof(double) * all.size(),
                               cudaMemcpyHostToDevice));
  }
  RMGTD_CUDA(ctx, cudaMemcpy(ctx->fld_nsamp, ns.data(), sizeof(int) * ctx->nrep,
                             cudaMemcpyHostToDevice));
  if (on != ctx->fld_on || regrow) {   // the step graph holds the field's kernels or not,
                                       // or their old buffer: rebuild it
    if (ctx->step_exec) cudaGraphExecDestroy(ctx->step_exec);
    if (ctx->step_graph) cudaGraphDestroy(ctx->step_graph);
    ctx->step_exec = nullptr;
    ctx->step_graph = nullptr;
  }
  ctx->fld_on = on;
  return RMGTD_OK;
}

int rmgtd_ground_state_info(rmgtd_ctx* ctx, int* iterations, double* drho, double* residual,
                            double* eps) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (ctx->opt.ground_state_scf <= 0)
    return set_error(ctx, RMGTD_ESTATE, "ground_state_info: created without the ground-state SCF");
  if (iterations) *iterations = ctx->gs_iters;
  if (drho) *drho = ctx->gs_err;
  if (residual) *residual = ctx->gs_resid;
  if (eps) std::copy(ctx->gs_eps.begin(), ctx->gs_eps.end(), eps);
  return RMGTD_OK;
}

int rmgtd_get_hartree_preconditioner(rmgtd_ctx* ctx, int* kind) {
  if (!ctx || !kind) return set_error(ctx, RMGTD_EINVAL, "get_hartree_preconditioner: NULL");
  *kind = hartree_precond_in_use(ctx);
  return RMGTD_OK;
}

int rmgtd_selftest_barrier_timeout(rmgtd_ctx* ctx, unsigned polls, int* status_out) {
  if (!ctx || !status_out) return set_error(ctx, RMGTD_EINVAL, "selftest: NULL argument");
  if (polls < 1 || polls > kSpinLimit)
    return set_error(ctx, RMGTD_EINVAL, "selftest: polls must be in 1 .. 20000000");
  unsigned* buf = (unsigned*)dev_alloc(ctx, 2 * sizeof(unsigned));
  if (!buf) return set_error(ctx, RMGTD_ENOMEM, "selftest buffer");
  int rc = RMGTD_OK;
  int st = 0;
  cudaError_t e = cudaMemsetAsync(buf, 0, 2 * sizeof(unsigned), ctx->stream);
  if (e == cudaSuccess) {
    k_barrier_timeout_probe<<<std::max(2, ctx->num_sms), 32, 0, ctx->stream>>>(
        buf, reinterpret_cast<int*>(buf + 1), polls);
    ++ctx->launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&st, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) rc = cuda_check(ctx, e, "selftest barrier time-out");
  dev_free(ctx, buf);
  if (rc == RMGTD_OK) *status_out = st;
  return rc;
}

int rmgtd_time(rmgtd_ctx* ctx, double* t, long long* steps) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (t) *t = ctx->t;
  if (steps) *steps = ctx->steps;
  return RMGTD_OK;
}

static const uint64_t kMagic = 0x32444d54474d52ull;  // "RMGTD2"

int rmgtd_save(rmgtd_ctx* ctx, const char* path) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (!path) return set_error(ctx, RMGTD_EINVAL, "save: path is NULL");
  if (ctx->opt.grid_basis) return set_error(ctx, RMGTD_ESTATE, "save: grid-basis context");
  const long NN = (long)ctx->N * ctx->N;
  const size_t mcount = (size_t)NN * ctx->nrep, gcount = (size_t)ctx->Ng * ctx->nrep;
  std::vector<double> buf(4 * mcount + gcount);
  const int rc = mixed_fields64(ctx);
  if (rc) return rc;
  double* parts[4] = {ctx->S0, ctx->A0, ctx->H0, ctx->Hm1};
  for (int i = 0; i < 4; ++i)
    RMGTD_CUDA(ctx, cudaMemcpyAsync(buf.data() + i * mcount, parts[i], sizeof(double) * mcount,
                                    cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(buf.data() + 4 * mcount, ctx->vh, sizeof(double) * gcount,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  FILE* fp = fopen(path, "wb");
  if (!fp) return set_error(ctx, RMGTD_EINVAL, std::string("save: cannot open ") + path);
  const int64_t hdr[7] = {ctx->nx, ctx->ny, ctx->nz, ctx->N, ctx->nrep, ctx->steps, ctx->mixed};
  bool ok = fwrite(&kMagic, sizeof(kMagic), 1, fp) == 1 && fwrite(hdr, sizeof(hdr), 1, fp) == 1 &&
            fwrite(&ctx->t, sizeof(double), 1, fp) == 1 &&
            fwrite(buf.data(), sizeof(double), buf.size(), fp) == buf.size();
  if (ok) {
    std::vector<double> vp(2 * gcount);
    RMGTD_CUDA(ctx, cudaMemcpy(vp.data(), ctx->vh_prev, sizeof(double) * gcount, cudaMemcpyDeviceToHost));
    RMGTD_CUDA(ctx, cudaMemcpy(vp.data() + gcount, ctx->vh_prev2, sizeof(double) * gcount,
                               cudaMemcpyDeviceToHost));
    ok = fwrite(vp.data(), sizeof(double), 2 * gcount, fp) == 2 * gcount;
  }
  if (ok && ctx->mixed) {
    std::vector<float> d32(3 * gcount);
    RMGTD_CUDA(ctx, cudaMemcpy(d32.data(), ctx->dvh32, sizeof(float) * gcount, cudaMemcpyDeviceToHost));
    RMGTD_CUDA(ctx, cudaMemcpy(d32.data() + gcount, ctx->dvh_prev32, sizeof(float) * gcount,
                               cudaMemcpyDeviceToHost));
    RMGTD_CUDA(ctx, cudaMemcpy(d32.data() + 2 * gcount, ctx->dvh_prev2_32, sizeof(float) * gcount,
                               cudaMemcpyDeviceToHost));
    ok = fwrite(d32.data(), sizeof(float), 3 * gcount, fp) == 3 * gcount;
  }
  if (ok && ctx->mixed && ctx->Sa) {   // anchors of the orbital-plane contractions
    std::vector<double> m(2 * mcount);
    std::vector<float> f(2 * gcount);
    RMGTD_CUDA(ctx, cudaMemcpy(m.data(), ctx->Sa, sizeof(double) * mcount, cudaMemcpyDeviceToHost));
    RMGTD_CUDA(ctx, cudaMemcpy(m.data() + mcount, ctx->Ha, sizeof(double) * mcount,
                               cudaMemcpyDeviceToHost));
    RMGTD_CUDA(ctx, cudaMemcpy(f.data(), ctx->rho_a32, sizeof(float) * gcount, cudaMemcpyDeviceToHost));
    RMGTD_CUDA(ctx, cudaMemcpy(f.data() + gcount, ctx->dv_a32, sizeof(float) * gcount,
                               cudaMemcpyDeviceToHost));
    ok = fwrite(m.data(), sizeof(double), 2 * mcount, fp) == 2 * mcount &&
         fwrite(f.data(), sizeof(float), 2 * gcount, fp) == 2 * gcount;
  }
  fclose(fp);
  if (!ok) return set_error(ctx, RMGTD_EINVAL, "save: write failed");
  return RMGTD_OK;
}

int rmgtd_load(rmgtd_ctx* ctx, const char* path) {
  if (!ctx) return set_error(nullptr, RMGTD_EINVAL, "ctx is NULL");
  if (!path) return set_error(ctx, RMGTD_EINVAL, "load: path is NULL");
  if (ctx->opt.grid_basis) return set_error(ctx, RMGTD_ESTATE, "load: grid-basis context");
  FILE* fp = fopen(path, "rb");
  if (!fp) return set_error(ctx, RMGTD_EINVAL, std::string("load: cannot open ") + path);
  uint64_t magic = 0;
  int64_t hdr[7];
  double t = 0;
  bool ok = fread(&magic, sizeof(magic), 1, fp) == 1 && fread(hdr, sizeof(hdr), 1, fp) == 1 &&
            fread(&t, sizeof(double), 1, fp) == 1;
  if (!ok || magic != kMagic || hdr[0] != ctx->nx || hdr[1] != ctx->ny || hdr[2] != ctx->nz ||
      hdr[3] != ctx->N || hdr[4] != ctx->nrep || hdr[6] != ctx->mixed) {
    fclose(fp);
    return set_error(ctx, RMGTD_EINVAL, "load: checkpoint does not match this context");
  }
  const long NN = (long)ctx->N * ctx->N;
  const size_t mcount = (size_t)NN * ctx->nrep, gcount = (size_t)ctx->Ng * ctx->nrep;
  std::vector<double> buf(4 * mcount + gcount);
  ok = fread(buf.data(), sizeof(double), buf.size(), fp) == buf.size();
  std::vector<double> vp(2 * gcount);
  if (ok) ok = fread(vp.data(), sizeof(double), 2 * gcount, fp) == 2 * gcount;
  std::vector<float> d32;
  if (ok && ctx->mixed) {
    d32.resize(3 * gcount);
    ok = fread(d32.data(), sizeof(float), 3 * gcount, fp) == 3 * gcount;
  }
  std::vector<double> am;
  std::vector<float> af;
  if (ok && ctx->mixed && ctx->Sa) {
    am.resize(2 * mcount);
    af.resize(2 * gcount);
    ok = fread(am.data(), sizeof(double), 2 * mcount, fp) == 2 * mcount &&
         fread(af.data(), sizeof(float), 2 * gcount, fp) == 2 * gcount;
  }
  fclose(fp);
  if (!ok) return set_error(ctx, RMGTD_EINVAL, "load: truncated checkpoint");
  RMGTD_CUDA(ctx, cudaMemcpy(ctx->vh_prev, vp.data(), sizeof(double) * gcount, cudaMemcpyHostToDevice));
  RMGTD_CUDA(ctx, cudaMemcpy(ctx->vh_prev2, vp.data() + gcount, sizeof(double) * gcount,
                             cudaMemcpyHostToDevice));
  if (ctx->mixed) {
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->dvh32, d32.data(), sizeof(float) * gcount, cudaMemcpyHostToDevice));
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->dvh_prev32, d32.data() + gcount, sizeof(float) * gcount,
                               cudaMemcpyHostToDevice));
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->dvh_prev2_32, d32.data() + 2 * gcount, sizeof(float) * gcount,
                               cudaMemcpyHostToDevice));
  }
  if (!am.empty()) {
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->Sa, am.data(), sizeof(double) * mcount, cudaMemcpyHostToDevice));
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->Ha, am.data() + mcount, sizeof(double) * mcount,
                               cudaMemcpyHostToDevice));
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->rho_a32, af.data(), sizeof(float) * gcount, cudaMemcpyHostToDevice));
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->dv_a32, af.data() + gcount, sizeof(float) * gcount,
                               cudaMemcpyHostToDevice));
  }
  double* parts[4] = {ctx->S0, ctx->A0, ctx->H0, ctx->Hm1};
  for (int i = 0; i < 4; ++i)
    RMGTD_CUDA(ctx, cudaMemcpyAsync(parts[i], buf.data() + i * mcount, sizeof(double) * mcount,
                                    cudaMemcpyHostToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->vh, buf.data() + 4 * mcount, sizeof(double) * gcount,
                                  cudaMemcpyHostToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->t = t;
  ctx->steps = hdr[5];
  {
    const long long sd = ctx->steps;
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->step_dev, &sd, sizeof(long long), cudaMemcpyHostToDevice));
  }
  if (ctx->Hm2)   // the quadratic seed restarts from H_-1
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Hm2, ctx->Hm1, sizeof(double) * mcount, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
  // observables need rho / eps_xc of the restored P; V_H is restored exactly (warm start)
  int rc = rho_dev(ctx, ctx->S0, ctx->rho, nullptr, ctx->nrep);
  if (rc) return rc;
  rc = launch_lda(ctx, ctx->rho, ctx->hartree_xc ? ctx->vh : nullptr, 0, ctx->vxc, ctx->exc,
                  ctx->vhxc, ctx->mixed ? ctx->dv32 : nullptr, ctx->Ng, nullptr, ctx->nrep,
                  ctx->Ng, ctx->hartree_xc);
  if (rc) return rc;
  ctx->fields_stale = 0;
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

}  // extern "C"
