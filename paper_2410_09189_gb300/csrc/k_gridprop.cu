// Propagation of the occupied orbitals on the grid: the complete-grid-basis limit of
// Algorithm 1 (Section 2.2: the propagation holds in any basis; the grid is the complete
// one).  P = sum_n f_n |psi_n><psi_n| is propagated by applying the series of Eq. 33 to the
// orbitals, psi^(k) = (-i dt / k) Hbar psi^(k-1), with Hbar = T + V_ion + V_NL +
// (V_0 + V_1)/2 + sum_q Ebar_q q, inside the same SCF loop on V = V_H + V_xc (in the grid
// basis H_new - H_1 is diagonal, so H_err = max|V_new - V_1|), then a Cholesky
// re-orthonormalisation in float64.  The kick is the pointwise phase e^{-i kappa q}.
//
// Layout: per replica the orbitals are planar complex, [2][nocc][Ng] (real plane, then
// imaginary plane), so the real stencil / KB operator applies to both planes as 2 nocc real
// columns.  Float64 throughout; the host drives the term and pass loops (one small read-back
// per term for the stopping test).
#include <cstring>
#include <utility>

#include "rmgtd_internal.cuh"

namespace rmgtd {

namespace {

__device__ __forceinline__ double coord_of(long g, int axis, int nx, int ny, int nz, double h) {
  const int i = axis == 0 ? (int)(g % nx) : axis == 1 ? (int)((g / nx) % ny) : (int)(g / ((long)nx * ny));
  const int n = axis == 0 ? nx : axis == 1 ? ny : nz;
  return axis_coord(i, n, h);
}

// psi_r = phi (real) for every replica
__global__ void k_gp_init(const double* __restrict__ phi, long plane, int nrep, double* __restrict__ psi) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < plane;
       e += (long)gridDim.x * blockDim.x) {
    const double v = phi[e];
    for (int r = 0; r < nrep; ++r) {
      psi[2 * r * plane + e] = v;
      psi[(2 * r + 1) * plane + e] = 0.0;
    }
  }
}

// psi <- e^{-i kappa q} psi on one replica's planes
__global__ void k_gp_kick(double* __restrict__ psi, int nocc, long Ng, int nx, int ny, int nz,
                          double h, int axis, double kappa) {
  const long plane = (long)nocc * Ng;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < plane;
       e += (long)gridDim.x * blockDim.x) {
    const double ph = -kappa * coord_of(e % Ng, axis, nx, ny, nz, h);
    double s, c;
    sincos(ph, &s, &c);
    const double re = psi[e], im = psi[plane + e];
    psi[e] = c * re - s * im;
    psi[plane + e] = s * re + c * im;
  }
}

// out = 2 a - b (V_1 <- 2 V_0 - V_-1, Algorithm 1 line 11 on the potential)
__global__ void k_gp_extrap(const double* __restrict__ a, const double* __restrict__ b,
                            double* __restrict__ out, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    out[e] = 2.0 * a[e] - b[e];
}

// vbar_r = (V0_r + V1_r)/2 + sum_q ebar_rq q
__global__ void k_gp_vbar(const double* __restrict__ v0, const double* __restrict__ v1,
                          const double* __restrict__ ebar, double* __restrict__ vbar, long Ng,
                          int nx, int ny, int nz, double h) {
  const int r = blockIdx.y;
  const double ex = ebar[3 * r], ey = ebar[3 * r + 1], ez = ebar[3 * r + 2];
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x) {
    const long o = r * Ng + g;
    double v = 0.5 * (v0[o] + v1[o]);
    if (ex != 0.0 || ey != 0.0 || ez != 0.0)
      v += ex * coord_of(g, 0, nx, ny, nz, h) + ey * coord_of(g, 1, nx, ny, nz, h) +
           ez * coord_of(g, 2, nx, ny, nz, h);
    vbar[o] = v;
  }
}

// one series term on one replica: t <- (-i c) Ht, psi1 += t, errbits <- max |t|^2
__global__ void k_gp_term(const double* __restrict__ Ht, double* __restrict__ t,
                          double* __restrict__ psi1, long plane, double c,
                          unsigned long long* __restrict__ errbits) {
  __shared__ double sh[32];
  double emax = 0.0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < plane;
       e += (long)gridDim.x * blockDim.x) {
    const double hr = Ht[e], hi = Ht[plane + e];
    const double tr = c * hi, ti = -c * hr;   // -i c (hr + i hi)
    t[e] = tr;
    t[plane + e] = ti;
    psi1[e] += tr;
    psi1[plane + e] += ti;
    emax = fmax(emax, tr * tr + ti * ti);
  }
  emax = block_max(emax, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(errbits, emax);
}

// rho_r = sum_n f_n |psi_n|^2
__global__ void k_gp_density(const double* __restrict__ psi, const double* __restrict__ f, int nocc,
                             long Ng, double* __restrict__ rho) {
  const int r = blockIdx.y;
  const long plane = (long)nocc * Ng;
  const double* p = psi + 2 * r * plane;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int n = 0; n < nocc; ++n) {
      const double re = p[(long)n * Ng + g], im = p[plane + (long)n * Ng + g];
      s = fma(f[n], re * re + im * im, s);
    }
    rho[r * Ng + g] = s;
  }
}

// errbits_r <- max |vnew - v1|; v1 <- vnew (replicas with active[r] = 0 untouched)
__global__ void k_gp_verr(const double* __restrict__ vnew, double* __restrict__ v1, long Ng,
                          const int* __restrict__ active, unsigned long long* __restrict__ errbits) {
  const int r = blockIdx.y;
  if (!active[r]) return;
  __shared__ double sh[32];
  double emax = 0.0;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x) {
    const long o = r * Ng + g;
    emax = fmax(emax, fabs(vnew[o] - v1[o]));
    v1[o] = vnew[o];
  }
  emax = block_max(emax, sh);
  if (threadIdx.x == 0) atomic_max_nonneg(&errbits[r], emax);
}

// Im part of the Gram: gim = Y - Y^T (Y_nm = h^3 sum Im psi_n Re psi_m)
__global__ void k_gp_antisym(int N, const double* __restrict__ Y, double* __restrict__ gim) {
  const long NN = (long)N * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < NN; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    gim[e] = Y[e] - Y[(long)j * N + i];
  }
}

// complex Cholesky G = L L^dagger (G Hermitian: real part gre, imaginary part gim), in place:
// the lower triangle of (gre, gim) becomes L; one block; status <- EINVAL on a non-positive
// pivot
__global__ void k_zcholesky(int N, double* __restrict__ gre, double* __restrict__ gim, int* status) {
  __shared__ double d;
  for (int k = 0; k < N; ++k) {
    if (threadIdx.x == 0) {
      const double v = gre[(long)k * N + k];
      if (!(v > 0.0)) atomicCAS(status, 0, (int)RMGTD_EINVAL);
      d = sqrt(fmax(v, 1e-300));
      gre[(long)k * N + k] = d;
      gim[(long)k * N + k] = 0.0;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < N; i += blockDim.x) {
      gre[(long)i * N + k] /= d;
      gim[(long)i * N + k] /= d;
    }
    __syncthreads();
    const long rem = (long)(N - k - 1);
    for (long e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = k + 1 + (int)(e / rem), j = k + 1 + (int)(e % rem);
      if (j <= i) {   // G_ij -= L_ik conj(L_jk)
        const double ar = gre[(long)i * N + k], ai = gim[(long)i * N + k];
        const double br = gre[(long)j * N + k], bi = gim[(long)j * N + k];
        gre[(long)i * N + j] -= ar * br + ai * bi;
        gim[(long)i * N + j] -= ai * br - ar * bi;
      }
    }
    __syncthreads();
  }
}

// psi_out = L^-1 psi_in per grid point (complex forward substitution, planar layout)
__global__ void k_gp_fsubst(int nocc, long Ng, const double* __restrict__ lre,
                            const double* __restrict__ lim, const double* __restrict__ in,
                            double* __restrict__ out) {
  const long plane = (long)nocc * Ng;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x) {
    for (int n = 0; n < nocc; ++n) {
      double sr = in[(long)n * Ng + g], si = in[plane + (long)n * Ng + g];
      for (int m = 0; m < n; ++m) {
        const double lr = lre[(long)n * nocc + m], li = lim[(long)n * nocc + m];
        const double yr = out[(long)m * Ng + g], yi = out[plane + (long)m * Ng + g];
        sr -= lr * yr - li * yi;
        si -= lr * yi + li * yr;
      }
      const double dn = lre[(long)n * nocc + n];
      out[(long)n * Ng + g] = sr / dn;
      out[plane + (long)n * Ng + g] = si / dn;
    }
  }
}

// per replica: [d_x, d_y, d_z, E_core, E_H, E_xc, N_e] partial sums over blocks (fixed order)
constexpr int kGpObs = 7;
__global__ void k_gp_obs(const double* __restrict__ psi, const double* __restrict__ hpsi,
                         const double* __restrict__ f, int nocc, long Ng, const double* __restrict__ rho,
                         const double* __restrict__ vh, const double* __restrict__ exc,
                         const double* __restrict__ rho_core, int nx, int ny, int nz, double h,
                         double* __restrict__ part) {
  const int r = blockIdx.y;
  const long plane = (long)nocc * Ng;
  const double* p = psi + 2 * r * plane;
  const double* hp = hpsi + 2 * r * plane;
  __shared__ double sh[32];
  double acc[kGpObs] = {0, 0, 0, 0, 0, 0, 0};
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x) {
    const double rg = rho[r * Ng + g];
    acc[0] += coord_of(g, 0, nx, ny, nz, h) * rg;
    acc[1] += coord_of(g, 1, nx, ny, nz, h) * rg;
    acc[2] += coord_of(g, 2, nx, ny, nz, h) * rg;
    double ec = 0.0;
    for (int n = 0; n < nocc; ++n) {
      const long o = (long)n * Ng + g;
      ec += f[n] * (p[o] * hp[o] + p[plane + o] * hp[plane + o]);
    }
    acc[3] += ec;
    acc[4] += 0.5 * rg * vh[r * Ng + g];
    acc[5] += (rg + (rho_core ? rho_core[g] : 0.0)) * exc[r * Ng + g];
    acc[6] += rg;
  }
  for (int q = 0; q < kGpObs; ++q) {
    const double v = block_sum(acc[q], sh);
    if (threadIdx.x == 0) part[((long)r * kGpObs + q) * gridDim.x + blockIdx.x] = v;
    __syncthreads();
  }
}

int gp_blocks(rmgtd_ctx* ctx, long n) {
  return (int)std::max<long>(1, std::min<long>(ceil_div(n, 256), 4L * ctx->num_sms));
}

}  // namespace

int gridprop_setup(rmgtd_ctx* ctx) {
  const int nocc = ctx->N, nrep = ctx->nrep;
  const long Ng = ctx->Ng, plane = (long)nocc * Ng;
  const size_t psz = sizeof(double) * 2 * plane * nrep;
  ctx->gp_psi = (double*)dev_alloc(ctx, psz);
  ctx->gp_psi1 = (double*)dev_alloc(ctx, psz);
  ctx->gp_t = (double*)dev_alloc(ctx, psz);
  ctx->gp_ht = (double*)dev_alloc(ctx, psz);
  const size_t vsz = sizeof(double) * Ng * nrep;
  ctx->gp_v0 = (double*)dev_alloc(ctx, vsz);
  ctx->gp_vm1 = (double*)dev_alloc(ctx, vsz);
  ctx->gp_v1 = (double*)dev_alloc(ctx, vsz);
  ctx->gp_vbar = (double*)dev_alloc(ctx, vsz);
  ctx->gp_ebar = (double*)dev_alloc(ctx, sizeof(double) * 3 * nrep);
  ctx->gp_active = (int*)dev_alloc(ctx, sizeof(int) * nrep);
  ctx->gp_gram = (double*)dev_alloc(ctx, sizeof(double) * 3 * (size_t)nocc * nocc);
  ctx->gp_obs = (double*)dev_alloc(ctx, sizeof(double) * kGpObs * nrep * 4L * ctx->num_sms);
  if (!ctx->gp_psi || !ctx->gp_psi1 || !ctx->gp_t || !ctx->gp_ht || !ctx->gp_v0 || !ctx->gp_vm1 ||
      !ctx->gp_v1 || !ctx->gp_vbar || !ctx->gp_ebar || !ctx->gp_active || !ctx->gp_gram ||
      !ctx->gp_obs)
    return set_error(ctx, RMGTD_ENOMEM, "grid propagation buffers");
  k_gp_init<<<gp_blocks(ctx, plane), 256, 0, ctx->stream>>>(ctx->phi, plane, nrep, ctx->gp_psi);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_init");
  // V_0 = V_-1 = V_H + V_xc of the starting density (computed by the set-up)
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_v0, ctx->vhxc, vsz, cudaMemcpyDeviceToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_vm1, ctx->vhxc, vsz, cudaMemcpyDeviceToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

int gridprop_kick(rmgtd_ctx* ctx, int rep, int axis, double kappa) {
  const long plane = (long)ctx->N * ctx->Ng;
  k_gp_kick<<<gp_blocks(ctx, plane), 256, 0, ctx->stream>>>(
      ctx->gp_psi + 2 * rep * plane, ctx->N, ctx->Ng, ctx->nx, ctx->ny, ctx->nz, ctx->h, axis, kappa);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_kick");
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;   // |psi|^2 unchanged: the fields stay as they are
}

// fields of the orbitals `psi` for every replica: rho, V_H, V_xc, eps_xc, V_Hxc (ctx arrays)
static int gp_fields(rmgtd_ctx* ctx, const double* psi) {
  const long Ng = ctx->Ng;
  k_gp_density<<<dim3(gp_blocks(ctx, Ng), ctx->nrep), 256, 0, ctx->stream>>>(psi, ctx->f_dev, ctx->N,
                                                                            Ng, ctx->rho);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_density");
  int rc = RMGTD_OK;
  if (ctx->hartree_xc) {
    rc = hartree_coop(ctx, ctx->rho, ctx->vh, nullptr, 0, ctx->nrep, 0);
    if (rc) return rc;
  }
  return launch_lda(ctx, ctx->rho, ctx->hartree_xc ? ctx->vh : nullptr, 0, ctx->vxc, ctx->exc,
                    ctx->vhxc, nullptr, Ng, nullptr, ctx->nrep, Ng, ctx->hartree_xc);
}

static int read_max(rmgtd_ctx* ctx, const unsigned long long* bits, int n, std::vector<double>& out) {
  std::vector<unsigned long long> h(n);
  RMGTD_CUDA(ctx, cudaMemcpyAsync(h.data(), bits, sizeof(unsigned long long) * n,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  out.resize(n);
  for (int i = 0; i < n; ++i) {
    double v;
    memcpy(&v, &h[i], sizeof(double));
    out[i] = v;
  }
  return RMGTD_OK;
}

// Cholesky re-orthonormalisation of psi1 into psi for one replica
static int gp_orthonormalize(rmgtd_ctx* ctx, int r) {
  const int N = ctx->N;
  const long plane = (long)N * ctx->Ng, NN = (long)N * N;
  const double* re = ctx->gp_psi1 + 2 * r * plane;
  const double* im = re + plane;
  double* gre = ctx->gp_gram;
  double* gim = gre + NN;
  double* y = gim + NN;
  // G_nm = h^3 sum psi_n conj(psi_m): Re = R R^T + I I^T, Im = Y - Y^T with Y = I R^T
  int rc = gram(ctx, re, re, nullptr, 0, 1, ctx->h3, nullptr, gre, nullptr, nullptr, 1, nullptr);
  if (!rc) rc = gram(ctx, im, im, nullptr, 0, 1, ctx->h3, gre, gre, nullptr, nullptr, 1, nullptr);
  if (!rc) rc = gram(ctx, im, re, nullptr, 0, 1, ctx->h3, nullptr, y, nullptr, nullptr, 0, nullptr);
  if (rc) return rc;
  k_gp_antisym<<<gp_blocks(ctx, NN), 256, 0, ctx->stream>>>(N, y, gim);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_antisym");
  k_zcholesky<<<1, 1024, 0, ctx->stream>>>(N, gre, gim, ctx->status);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_zcholesky");
  k_gp_fsubst<<<gp_blocks(ctx, ctx->Ng), 256, 0, ctx->stream>>>(N, ctx->Ng, gre, gim, re,
                                                               ctx->gp_psi + 2 * r * plane);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_fsubst");
  return RMGTD_OK;
}

int gridprop_step(rmgtd_ctx* ctx, rmgtd_stats* st) {
  const int nrep = ctx->nrep, N = ctx->N;
  const long Ng = ctx->Ng, plane = (long)N * Ng;
  const double dt = ctx->opt.dt;
  const double thr2 = ctx->opt.dP_thrs * ctx->opt.dP_thrs;
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  // the step's mean field per replica from the host samples E(j dt) (zero past them)
  {
    std::vector<double> eb(3 * nrep, 0.0);
    const long long k = ctx->gp_steps;
    for (int r = 0; r < nrep; ++r) {
      const auto& E = ctx->fld_host[r];
      const long long ns = (long long)E.size() / 3;
      for (int q = 0; q < 3; ++q) {
        const double e0 = k < ns ? E[3 * k + q] : 0.0, e1 = k + 1 < ns ? E[3 * (k + 1) + q] : 0.0;
        eb[3 * r + q] = 0.5 * (e0 + e1);
      }
    }
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_ebar, eb.data(), sizeof(double) * 3 * nrep,
                                    cudaMemcpyHostToDevice, ctx->stream));
  }
  const int vb = gp_blocks(ctx, Ng * nrep);
  k_gp_extrap<<<vb, 256, 0, ctx->stream>>>(ctx->gp_v0, ctx->gp_vm1, ctx->gp_v1, Ng * nrep);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_extrap");
  std::vector<int> active(nrep, 1), passes(nrep, 0), tmax(nrep, 0), tsum(nrep, 0), status(nrep, 0);
  std::vector<double> herr(nrep, 0.0), m;
  bool any = true;
  for (int pass = 1; pass <= ctx->opt.max_scf && any; ++pass) {
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_active, active.data(), sizeof(int) * nrep,
                                    cudaMemcpyHostToDevice, ctx->stream));
    k_gp_vbar<<<dim3(gp_blocks(ctx, Ng), nrep), 256, 0, ctx->stream>>>(
        ctx->gp_v0, ctx->gp_v1, ctx->gp_ebar, ctx->gp_vbar, Ng, ctx->nx, ctx->ny, ctx->nz, ctx->h);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_vbar");
    // the orbital series of every active replica
    std::vector<int> series(nrep, 0);
    for (int r = 0; r < nrep; ++r) {
      if (!active[r]) continue;
      series[r] = 1;
      const size_t b = sizeof(double) * 2 * plane;
      RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_psi1 + 2 * r * plane, ctx->gp_psi + 2 * r * plane, b,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
      RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_t + 2 * r * plane, ctx->gp_psi + 2 * r * plane, b,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    }
    int k = 0;
    for (bool more = true; more;) {
      ++k;
      RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->errbits, 0, sizeof(unsigned long long) * nrep, ctx->stream));
      for (int r = 0; r < nrep; ++r) {
        if (!series[r]) continue;
        int rc = apply_h_dev(ctx, ctx->gp_t + 2 * r * plane, ctx->gp_ht + 2 * r * plane, 2 * N,
                             RMGTD_F64, ctx->gp_vbar + r * Ng);
        if (rc) return rc;
        k_gp_term<<<gp_blocks(ctx, plane), 256, 0, ctx->stream>>>(
            ctx->gp_ht + 2 * r * plane, ctx->gp_t + 2 * r * plane, ctx->gp_psi1 + 2 * r * plane,
            plane, dt / k, ctx->errbits + r);
        ++ctx->launches;
        RMGTD_LAUNCH(ctx, "k_gp_term");
      }
      int rc = read_max(ctx, ctx->errbits, nrep, m);
      if (rc) return rc;
      more = false;
      for (int r = 0; r < nrep; ++r) {
        if (!series[r]) continue;
        if (!(m[r] <= 1e300)) {
          status[r] = RMGTD_EDIVERGED;
          series[r] = 0;
        } else if (m[r] <= thr2) {
          series[r] = 0;
        } else if (k >= ctx->opt.max_terms) {
          status[r] = RMGTD_ENOTCONVERGED;
          series[r] = 0;
        } else {
          more = true;
        }
        if (!series[r]) {
          tmax[r] = std::max(tmax[r], k);
          tsum[r] += k;
        }
      }
    }
    for (int r = 0; r < nrep; ++r)
      if (status[r]) active[r] = 0;
    // V_new of the propagated orbitals; H_err = max|V_new - V_1|
    int rc = gp_fields(ctx, ctx->gp_psi1);
    if (rc) return rc;
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_active, active.data(), sizeof(int) * nrep,
                                    cudaMemcpyHostToDevice, ctx->stream));
    RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->errbits, 0, sizeof(unsigned long long) * nrep, ctx->stream));
    k_gp_verr<<<dim3(gp_blocks(ctx, Ng), nrep), 256, 0, ctx->stream>>>(ctx->vhxc, ctx->gp_v1, Ng,
                                                                       ctx->gp_active, ctx->errbits);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_verr");
    rc = read_max(ctx, ctx->errbits, nrep, m);
    if (rc) return rc;
    any = false;
    for (int r = 0; r < nrep; ++r) {
      if (!active[r]) continue;
      passes[r] = pass;
      herr[r] = m[r];
      if (!(m[r] <= 1e300)) {
        status[r] = RMGTD_EDIVERGED;
        active[r] = 0;
      } else if (m[r] <= ctx->opt.H_thrs) {
        active[r] = 0;
      } else if (pass == ctx->opt.max_scf) {
        status[r] = RMGTD_ENOTCONVERGED;
        active[r] = 0;
      } else {
        any = true;
      }
    }
  }
  int first = 0;
  for (int r = 0; r < nrep; ++r) {
    if (st) {
      st[r].passes = passes[r];
      st[r].terms_max = tmax[r];
      st[r].terms_sum = tsum[r];
      st[r].status = status[r];
      st[r].H_err = herr[r];
    }
    if (status[r] && !first) first = status[r];
  }
  if (first) {   // keep the last completed state: psi and the potential history are untouched
    int rc = gp_fields(ctx, ctx->gp_psi);
    if (rc) return rc;
    return set_error(ctx, first, "grid propagation step " + std::to_string(ctx->gp_steps) +
                                     " failed with status " + std::to_string(first));
  }
  for (int r = 0; r < nrep; ++r) {
    int rc = gp_orthonormalize(ctx, r);
    if (rc) return rc;
  }
  int cst = 0;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(&cst, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  // V_-1 <- V_0, V_0 <- V_1 (rotate the buffers)
  std::swap(ctx->gp_vm1, ctx->gp_v0);
  std::swap(ctx->gp_v0, ctx->gp_v1);
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (cst) return set_error(ctx, RMGTD_EDIVERGED, "grid propagation: overlap lost positivity");
  ++ctx->gp_steps;
  return RMGTD_OK;
}

// observables of every replica's current orbitals: fields re-evaluated from their density
int gridprop_observables(rmgtd_ctx* ctx) {
  const int nrep = ctx->nrep, N = ctx->N;
  const long Ng = ctx->Ng, plane = (long)N * Ng;
  int rc = gp_fields(ctx, ctx->gp_psi);
  if (rc) return rc;
  for (int r = 0; r < nrep; ++r) {   // H_core psi (no V_Hxc) into the scratch planes
    rc = apply_h_dev(ctx, ctx->gp_psi + 2 * r * plane, ctx->gp_ht + 2 * r * plane, 2 * N, RMGTD_F64,
                     nullptr);
    if (rc) return rc;
  }
  const int blocks = gp_blocks(ctx, Ng);
  k_gp_obs<<<dim3(blocks, nrep), 256, 0, ctx->stream>>>(
      ctx->gp_psi, ctx->gp_ht, ctx->f_dev, N, Ng, ctx->rho, ctx->vh, ctx->exc, ctx->rho_core,
      ctx->nx, ctx->ny, ctx->nz, ctx->h, ctx->gp_obs);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_obs");
  std::vector<double> part((size_t)kGpObs * nrep * blocks);
  RMGTD_CUDA(ctx, cudaMemcpyAsync(part.data(), ctx->gp_obs, sizeof(double) * part.size(),
                                  cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->gp_obs_host.assign((size_t)kGpObs * nrep, 0.0);
  for (int r = 0; r < nrep; ++r)
    for (int q = 0; q < kGpObs; ++q) {
      double s = 0.0;
      for (int b = 0; b < blocks; ++b) s += part[((size_t)r * kGpObs + q) * blocks + b];
      ctx->gp_obs_host[(size_t)r * kGpObs + q] = ctx->h3 * s;
    }
  return RMGTD_OK;
}

// d_q, E and N_e of replica `rep` from the last gridprop_observables
void gridprop_read(const rmgtd_ctx* ctx, int rep, double* d3, double* E, double* ne) {
  const double* o = ctx->gp_obs_host.data() + (size_t)rep * kGpObs;
  if (d3) {
    d3[0] = o[0];
    d3[1] = o[1];
    d3[2] = o[2];
  }
  if (E) *E = o[3] + o[4] + o[5] + ctx->E_ion;
  if (ne) *ne = o[6];
}

}  // namespace rmgtd
