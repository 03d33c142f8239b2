// Ground state on the GPU (Algorithm 1's ground state): the self-consistent Kohn-Sham orbitals that
// define the active space, computed from the starting orbitals before the set-up continues.
//
// Eigensolver: Chebyshev-filtered subspace iteration on a block of N + nb orbitals (nb buffer
// vectors, so the N-th eigenpair converges at the rate of the (N + nb)-th).  Per SCF iteration:
// the degree-m Chebyshev polynomial of H (T + V_ion + V_NL + V_Hxc(rho_in)) that damps the
// interval [a, b] above the block's highest Ritz value a (b bounds the spectrum: the
// stencil's Gershgorin bound, max V and the KB energies) is applied to the block, in the
// scaled three-term form that keeps the wanted components O(1); the block is orthonormalised
// by Cholesky-QR (float64) and rotated to the Ritz vectors of h^3 X^T H X (Jacobi on the
// device); rho_out = sum_n f_n x_n^2 of the N lowest; the density is Pulay-mixed (history of
// six, as the oracle's SCF) and V_Hxc rebuilt.  Converged when max|rho_out - rho_in| and the
// largest Ritz-pair residual max_g |H x_n - theta_n x_n| (n < N) are below the tolerance.
// Every operator application is the library's stencil / KB kernels; the small dense algebra
// (Gram, Cholesky, Jacobi, rotation) runs on the device, the Pulay coefficients on the host.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "jacobi.cuh"
#include "rmgtd_internal.cuh"

namespace rmgtd {

namespace {

int gs_blocks(rmgtd_ctx* ctx, long n) {
  return (int)std::max<long>(1, std::min<long>(ceil_div(n, 256), 4L * ctx->num_sms));
}

// Symmetric eigenpairs of A (n x n, n <= 1024) in one block: eigenvalues ascending in w, the
// eigenvector of w[k] in column k of Q (row-major).  work: 2 n^2 doubles.
__global__ void __launch_bounds__(1024)
k_sym_eig(int n, const double* __restrict__ A, double* __restrict__ work, double* __restrict__ w,
          double* __restrict__ Q) {
  __shared__ int pp[513], qq[513];
  __shared__ double cc[513], ss[513];
  __shared__ double sh[32];
  __shared__ int ord[1024];
  __shared__ double stop;
  const long nn = (long)n * n;
  double* Aw = work;
  double* V = work + nn;
  for (long e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    Aw[e] = 0.5 * (A[e] + A[(long)j * n + i]);   // symmetrised
    V[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_sweeps(n, Aw, V, pp, qq, cc, ss, sh, &stop);
  if (threadIdx.x == 0) {   // ascending order (insertion sort)
    for (int i = 0; i < n; ++i) ord[i] = i;
    for (int i = 1; i < n; ++i) {
      const int o = ord[i];
      const double d = Aw[(long)o * n + o];
      int j = i - 1;
      while (j >= 0 && Aw[(long)ord[j] * n + ord[j]] > d) {
        ord[j + 1] = ord[j];
        --j;
      }
      ord[j + 1] = o;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) w[k] = Aw[(long)ord[k] * n + ord[k]];
  for (long e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = (int)(e / n), k = (int)(e % n);
    Q[e] = V[(long)i * n + ord[k]];
  }
}

// Xout_k = sum_m Q[m][k] Xin_m (columns of length Ng), one thread per point; Q in shared memory
// in slices of kRotM rows
constexpr int kRotM = 32;
__global__ void __launch_bounds__(256)
k_rotate(int n, long Ng, const double* __restrict__ Q, const double* __restrict__ Xin,
         double* __restrict__ Xout) {
  __shared__ double sq[kRotM][kRotM];
  const long g = blockIdx.x * (long)blockDim.x + threadIdx.x;
  for (int k0 = 0; k0 < n; k0 += kRotM) {
    double acc[kRotM];
#pragma unroll
    for (int kk = 0; kk < kRotM; ++kk) acc[kk] = 0.0;
    for (int m0 = 0; m0 < n; m0 += kRotM) {
      __syncthreads();
      for (int e = threadIdx.x; e < kRotM * kRotM; e += blockDim.x) {
        const int mm = e / kRotM, kk = e % kRotM;
        sq[mm][kk] = (m0 + mm < n && k0 + kk < n) ? Q[(long)(m0 + mm) * n + k0 + kk] : 0.0;
      }
      __syncthreads();
      if (g < Ng) {
        const int mn = min(kRotM, n - m0);
        for (int mm = 0; mm < mn; ++mm) {
          const double x = Xin[(long)(m0 + mm) * Ng + g];
#pragma unroll
          for (int kk = 0; kk < kRotM; ++kk) acc[kk] = fma(sq[mm][kk], x, acc[kk]);
        }
      }
    }
    if (g < Ng) {
      const int kn = min(kRotM, n - k0);
      for (int kk = 0; kk < kn; ++kk) Xout[(long)(k0 + kk) * Ng + g] = acc[kk];
    }
  }
}

// out = s1 (HY - c Y) - s2 X   (one step of the scaled Chebyshev recurrence)
__global__ void k_cheb(long n, const double* __restrict__ HY, const double* __restrict__ Y,
                       const double* __restrict__ X, double c, double s1, double s2,
                       double* __restrict__ out) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    out[e] = s1 * (HY[e] - c * Y[e]) - (X ? s2 * X[e] : 0.0);
}

// rho = sum_{n < N} f_n x_n^2
__global__ void k_gs_density(int N, long Ng, const double* __restrict__ X, const double* __restrict__ f,
                             double* __restrict__ rho) {
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int n = 0; n < N; ++n) {
      const double x = X[(long)n * Ng + g];
      s = fma(f[n], x * x, s);
    }
    rho[g] = s;
  }
}

// per-block partial sums of a_i . b for up to 8 vectors a_i against b, and the max |a_0 - b|
// (slot 8): [block][9]
__global__ void k_gs_dots(int na, long n, const double* __restrict__ a, long astride,
                          const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const double be = b[e];
    for (int i = 0; i < na; ++i) acc[i] = fma(a[i * astride + e], be, acc[i]);
    acc[8] = fmax(acc[8], fabs(a[e] - be));
  }
  for (int i = 0; i < 9; ++i) {
    const double v = (i < 8) ? block_sum(acc[i], sh) : block_max(acc[i], sh);
    if (threadIdx.x == 0) part[(long)blockIdx.x * 9 + i] = v;
    __syncthreads();
  }
}

// out = max(0, sum_i c_i (rin_i + alpha res_i)) over the Pulay history
__global__ void k_gs_pulay(int m, long n, const double* __restrict__ rin, const double* __restrict__ res,
                           long stride, const double* __restrict__ coef, double alpha,
                           double* __restrict__ out) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int i = 0; i < m; ++i) v += coef[i] * (rin[i * stride + e] + alpha * res[i * stride + e]);
    out[e] = fmax(v, 0.0);
  }
}

// max over g of |HX_n - theta_n X_n| for each n < N (block per column)
__global__ void k_gs_resid(long Ng, const double* __restrict__ HX, const double* __restrict__ X,
                           const double* __restrict__ theta, double* __restrict__ out) {
  __shared__ double sh[32];
  const int n = blockIdx.x;
  double m = 0.0;
  for (long g = threadIdx.x; g < Ng; g += blockDim.x)
    m = fmax(m, fabs(HX[(long)n * Ng + g] - theta[n] * X[(long)n * Ng + g]));
  m = block_max(m, sh);
  if (threadIdx.x == 0) out[n] = m;
}

// per-block maxima of V_ion + V_Hxc (the spectrum bound)
__global__ void k_gs_vmax(long Ng, const double* __restrict__ a, const double* __restrict__ b,
                          double* __restrict__ part) {
  __shared__ double sh[32];
  double m = -1e300;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x)
    m = fmax(m, a[g] + b[g]);
  m = block_max(m, sh);   // (max with 0: still an upper bound, which is all the filter needs)
  if (threadIdx.x == 0) part[blockIdx.x] = m;
}

// deterministic pseudo-random start vectors (a counter hash: splitmix64 of the index)
__global__ void k_gs_noise(long n, unsigned long long seed, double* __restrict__ out) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(e + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    out[e] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

}  // namespace

namespace {

constexpr int kGsDegree = 12;     // Chebyshev filter degree per SCF iteration
constexpr double kGsMix = 0.4;    // Pulay mixing parameter (as the oracle's SCF)

struct GsWork {
  int N = 0, nb = 0, nt = 0;   // occupied + virtual, buffer, block
  long Ng = 0;
  double *X = nullptr, *Y = nullptr, *HY = nullptr, *Xo = nullptr, *T = nullptr;
  double *Hs = nullptr, *eigw = nullptr, *Q = nullptr, *theta = nullptr, *resid = nullptr;
  double *rho_in = nullptr, *rho_out = nullptr, *hist_in = nullptr, *hist_res = nullptr;
  double *part = nullptr, *coef = nullptr;
  int nblk = 0;
};

// H X for the block (T + V_ion + V_NL + V_Hxc of the current density)
int gs_apply(rmgtd_ctx* ctx, GsWork& w, const double* x, double* hx) {
  return apply_h_dev(ctx, x, hx, w.nt, RMGTD_F64, ctx->vhxc);
}

// h^3 A^T B for nt columns (the context's N is the block size during the solve)
int gs_gram(rmgtd_ctx* ctx, const double* A, const double* B, double* out, int sym) {
  return gram(ctx, A, B, nullptr, 0, 1, ctx->h3, nullptr, out, nullptr, nullptr, sym, nullptr);
}

// Rayleigh-Ritz: X <- X Q (Ritz vectors, ascending), theta; HX rotated alike into T
int gs_rayleigh_ritz(rmgtd_ctx* ctx, GsWork& w, bool want_resid) {
  int rc = gs_apply(ctx, w, w.X, w.HY);
  if (!rc) rc = gs_gram(ctx, w.X, w.HY, w.Hs, 0);
  if (rc) return rc;
  k_sym_eig<<<1, 1024, 0, ctx->stream>>>(w.nt, w.Hs, w.eigw, w.theta, w.Q);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_sym_eig");
  const int rb = (int)ceil_div(w.Ng, 256);
  k_rotate<<<rb, 256, 0, ctx->stream>>>(w.nt, w.Ng, w.Q, w.X, w.T);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_rotate");
  std::swap(w.X, w.T);
  if (want_resid) {
    k_rotate<<<rb, 256, 0, ctx->stream>>>(w.nt, w.Ng, w.Q, w.HY, w.T);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_rotate");
    k_gs_resid<<<w.N, 256, 0, ctx->stream>>>(w.Ng, w.T, w.X, w.theta, w.resid);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gs_resid");
  }
  return RMGTD_OK;
}

// Cholesky-QR of the block: X <- L^-1 X with h^3 X X^T = L L^T
int gs_orthonormalize(rmgtd_ctx* ctx, GsWork& w) {
  int rc = gs_gram(ctx, w.X, w.X, w.Hs, 1);
  if (rc) return rc;
  k_cholesky<<<1, 1024, 0, ctx->stream>>>(w.nt, w.Hs, ctx->status);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_cholesky");
  return forward_subst(ctx, w.nt, w.Hs, w.X, w.T);
}

// V_Hxc of rho (replica 0's field buffers)
int gs_potential(rmgtd_ctx* ctx, const double* rho) {
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->rho, rho, sizeof(double) * ctx->Ng, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  if (ctx->hartree_xc) {
    const int rc = hartree_coop(ctx, ctx->rho, ctx->vh, nullptr, 0, 1, 0);
    if (rc) return rc;
  }
  return launch_lda(ctx, ctx->rho, ctx->hartree_xc ? ctx->vh : nullptr, 0, ctx->vxc, ctx->exc,
                    ctx->vhxc, nullptr, ctx->Ng, nullptr, 1, ctx->Ng, ctx->hartree_xc);
}

// the block's dot products a_i . b (i < na, rows of stride astride) and max|a_0 - b|
int gs_dots(rmgtd_ctx* ctx, GsWork& w, int na, const double* a, long astride, const double* b,
            double* out /* [9] */) {
  k_gs_dots<<<w.nblk, 256, 0, ctx->stream>>>(na, w.Ng, a, astride, b, w.part);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gs_dots");
  std::vector<double> p((size_t)w.nblk * 9);
  RMGTD_CUDA(ctx, cudaMemcpyAsync(p.data(), w.part, sizeof(double) * p.size(), cudaMemcpyDeviceToHost,
                                  ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < 9; ++i) out[i] = 0.0;
  for (int b2 = 0; b2 < w.nblk; ++b2)
    for (int i = 0; i < 9; ++i)
      out[i] = (i < 8) ? out[i] + p[(size_t)b2 * 9 + i] : std::max(out[i], p[(size_t)b2 * 9 + i]);
  return RMGTD_OK;
}

// solve the bordered Pulay system [B 1; 1 0][c; l] = [0; 1] (Gaussian elimination with
// partial pivoting; a singular system falls back to the newest entry)
std::vector<double> pulay_coefficients(const std::vector<std::vector<double>>& B) {
  const int m = (int)B.size(), n = m + 1;
  std::vector<double> a((size_t)n * (n + 1), 0.0);
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) a[(size_t)i * (n + 1) + j] = B[i][j];
    a[(size_t)i * (n + 1) + m] = 1.0;
    a[(size_t)m * (n + 1) + i] = 1.0;
  }
  a[(size_t)m * (n + 1) + n] = 1.0;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(a[(size_t)i * (n + 1) + k]) > std::fabs(a[(size_t)piv * (n + 1) + k])) piv = i;
    if (std::fabs(a[(size_t)piv * (n + 1) + k]) < 1e-300) {
      std::vector<double> c(m, 0.0);
      c[m - 1] = 1.0;
      return c;
    }
    for (int j = 0; j <= n; ++j) std::swap(a[(size_t)k * (n + 1) + j], a[(size_t)piv * (n + 1) + j]);
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = a[(size_t)i * (n + 1) + k] / a[(size_t)k * (n + 1) + k];
      for (int j = k; j <= n; ++j) a[(size_t)i * (n + 1) + j] -= f * a[(size_t)k * (n + 1) + j];
    }
  }
  std::vector<double> c(m);
  for (int i = 0; i < m; ++i) c[i] = a[(size_t)i * (n + 1) + n] / a[(size_t)i * (n + 1) + i];
  return c;
}

}  // namespace

int ground_state_scf(rmgtd_ctx* ctx) {
  const int N = ctx->N, maxit = ctx->opt.ground_state_scf;
  const double tol = ctx->opt.ground_state_tol > 0 ? ctx->opt.ground_state_tol : 1e-8;
  GsWork w;
  w.N = N;
  w.nb = std::max(4, (N + 7) / 8);
  w.nt = N + w.nb;
  w.Ng = ctx->Ng;
  if (w.nt > 1024) return set_error(ctx, RMGTD_EINVAL, "ground state: N + buffer must be <= 1024");
  const long Ng = w.Ng, nt = w.nt;
  const size_t bsz = sizeof(double) * nt * Ng;
  std::vector<void*> mine;
  auto A = [&](size_t b) {
    void* p = dev_alloc(ctx, b);
    mine.push_back(p);
    return (double*)p;
  };
  w.X = A(bsz);
  w.Y = A(bsz);
  w.HY = A(bsz);
  w.Xo = A(bsz);
  w.T = A(bsz);
  w.Hs = A(sizeof(double) * nt * nt);
  w.eigw = A(sizeof(double) * 2 * nt * nt);
  w.Q = A(sizeof(double) * nt * nt);
  w.theta = A(sizeof(double) * nt);
  w.resid = A(sizeof(double) * N);
  w.rho_in = A(sizeof(double) * Ng);
  w.rho_out = A(sizeof(double) * Ng);
  w.hist_in = A(sizeof(double) * 6 * Ng);
  w.hist_res = A(sizeof(double) * 6 * Ng);
  w.nblk = gs_blocks(ctx, Ng);
  w.part = A(sizeof(double) * 9 * w.nblk);
  w.coef = A(sizeof(double) * 8);
  struct Cleanup {
    rmgtd_ctx* c;
    int N;
    std::vector<void*>* bufs;
    ~Cleanup() {
      c->N = N;
      cudaStreamSynchronize(c->stream);
      for (void* p : *bufs) dev_free(c, p);
    }
  } cleanup{ctx, N, &mine};
  for (void* p : mine)
    if (!p) return set_error(ctx, RMGTD_ENOMEM, "ground state buffers");
  const int eb = gs_blocks(ctx, nt * Ng);
  // an empty Pulay history reads as zeros (its coefficients are zero)
  RMGTD_CUDA(ctx, cudaMemsetAsync(w.hist_in, 0, sizeof(double) * 6 * Ng, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(w.hist_res, 0, sizeof(double) * 6 * Ng, ctx->stream));
  // the block: the N starting orbitals and nb deterministic noise vectors, orthonormalised
  RMGTD_CUDA(ctx, cudaMemcpyAsync(w.X, ctx->phi, sizeof(double) * N * Ng, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  k_gs_noise<<<eb, 256, 0, ctx->stream>>>((long)w.nb * Ng, 0x5EED5EEDull, w.X + (long)N * Ng);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gs_noise");
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  k_gs_density<<<w.nblk, 256, 0, ctx->stream>>>(N, Ng, ctx->phi, ctx->f_dev, w.rho_in);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gs_density");
  ctx->N = (int)nt;   // gram() and the KB buffers size by the context's N during the solve
  int rc = gs_orthonormalize(ctx, w);
  if (!rc) rc = gs_potential(ctx, w.rho_in);
  if (!rc) rc = gs_rayleigh_ritz(ctx, w, false);
  if (rc) return rc;
  // spectrum bound: the stencil's Gershgorin bound, max V, the positive KB energies
  double tb = std::fabs(fd_coef(0));
  for (int m = 1; m <= kFdRadius; ++m) tb += 2.0 * std::fabs(fd_coef(m));
  tb *= 1.5 / (ctx->h * ctx->h);
  double ekb = 0.0;
  for (double e : ctx->h_Ekb) ekb += std::max(e, 0.0);
  std::vector<double> theta(nt), resid(N), hb(9);
  std::vector<std::vector<double>> B;
  int nh = 0, head = 0;
  bool done = false;
  int it = 0;
  double err = 0.0, rmax = 0.0;
  for (it = 1; it <= maxit && !done; ++it) {
    RMGTD_CUDA(ctx, cudaMemcpyAsync(theta.data(), w.theta, sizeof(double) * nt, cudaMemcpyDeviceToHost,
                                    ctx->stream));
    k_gs_vmax<<<w.nblk, 256, 0, ctx->stream>>>(Ng, ctx->vion, ctx->vhxc, w.part);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gs_vmax");
    std::vector<double> vm(w.nblk);
    RMGTD_CUDA(ctx, cudaMemcpyAsync(vm.data(), w.part, sizeof(double) * w.nblk, cudaMemcpyDeviceToHost,
                                    ctx->stream));
    RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const double vmax = *std::max_element(vm.begin(), vm.end());
    const double b = tb + vmax + ekb, a = theta[nt - 1], aL = theta[0];
    if (!(b > a) || !(a > aL)) return set_error(ctx, RMGTD_EDIVERGED, "ground state: bad spectrum bounds");
    // Chebyshev filter of degree kGsDegree on [a, b], scaled at aL
    const double e = 0.5 * (b - a), c = 0.5 * (b + a);
    double sigma = e / (aL - c);
    const double tau = 2.0 / sigma;
    double* P0 = w.X;    // p_{k-1}(H) X
    double* P1 = w.Y;    // p_k(H) X
    double* P2 = w.Xo;   // scratch
    rc = gs_apply(ctx, w, P0, w.HY);
    if (rc) return rc;
    k_cheb<<<eb, 256, 0, ctx->stream>>>(nt * Ng, w.HY, P0, nullptr, c, sigma / e, 0.0, P1);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_cheb");
    for (int k = 2; k <= kGsDegree; ++k) {
      const double sn = 1.0 / (tau - sigma);
      rc = gs_apply(ctx, w, P1, w.HY);
      if (rc) return rc;
      k_cheb<<<eb, 256, 0, ctx->stream>>>(nt * Ng, w.HY, P1, P0, c, 2.0 * sn / e, sigma * sn, P2);
      ++ctx->launches;
      RMGTD_LAUNCH(ctx, "k_cheb");
      double* t = P0;
      P0 = P1;
      P1 = P2;
      P2 = t;
      sigma = sn;
    }
    // the filtered block becomes X (the other two buffers stay scratch)
    w.X = P1;
    w.Y = P0;
    w.Xo = P2;
    rc = gs_orthonormalize(ctx, w);
    if (!rc) rc = gs_rayleigh_ritz(ctx, w, true);
    if (rc) return rc;
    k_gs_density<<<w.nblk, 256, 0, ctx->stream>>>(N, Ng, w.X, ctx->f_dev, w.rho_out);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gs_density");
    RMGTD_CUDA(ctx, cudaMemcpyAsync(resid.data(), w.resid, sizeof(double) * N, cudaMemcpyDeviceToHost,
                                    ctx->stream));
    rc = gs_dots(ctx, w, 0, w.rho_out, Ng, w.rho_in, hb.data());   // max|rho_out - rho_in|
    if (rc) return rc;
    err = hb[8];
    rmax = *std::max_element(resid.begin(), resid.end());
    if (!std::isfinite(err) || !std::isfinite(rmax))
      return set_error(ctx, RMGTD_EDIVERGED, "ground state: non-finite density or residual");
    if (err <= tol && rmax <= tol) {
      done = true;
      break;
    }
    if (!ctx->hartree_xc) {   // independent electrons: the potential does not depend on rho
      RMGTD_CUDA(ctx, cudaMemcpyAsync(w.rho_in, w.rho_out, sizeof(double) * Ng, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
      continue;
    }
    // Pulay mixing of the residual rho_out - rho_in (history of six, oldest replaced)
    double* slot_in = w.hist_in + (long)head * Ng;
    double* slot_res = w.hist_res + (long)head * Ng;
    RMGTD_CUDA(ctx, cudaMemcpyAsync(slot_in, w.rho_in, sizeof(double) * Ng, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
    k_cheb<<<w.nblk, 256, 0, ctx->stream>>>(Ng, w.rho_out, w.rho_in, nullptr, 1.0, 1.0, 0.0, slot_res);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_cheb");
    nh = std::min(nh + 1, 6);
    head = (head + 1) % 6;
    // the history in age order: oldest first
    std::vector<int> order(nh);
    for (int i = 0; i < nh; ++i) order[i] = (head - nh + i + 6) % 6;
    B.assign(nh, std::vector<double>(nh, 0.0));
    for (int j = 0; j < nh; ++j) {
      rc = gs_dots(ctx, w, 6, w.hist_res, Ng, w.hist_res + (long)order[j] * Ng, hb.data());
      if (rc) return rc;
      for (int i = 0; i < nh; ++i) B[i][j] = hb[order[i]];
    }
    const std::vector<double> cf = pulay_coefficients(B);
    std::vector<double> c6(6, 0.0);
    for (int i = 0; i < nh; ++i) c6[order[i]] = cf[i];
    RMGTD_CUDA(ctx, cudaMemcpyAsync(w.coef, c6.data(), sizeof(double) * 6, cudaMemcpyHostToDevice,
                                    ctx->stream));
    k_gs_pulay<<<w.nblk, 256, 0, ctx->stream>>>(6, Ng, w.hist_in, w.hist_res, Ng, w.coef, kGsMix,
                                                w.rho_in);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gs_pulay");
    rc = gs_potential(ctx, w.rho_in);
    if (rc) return rc;
  }
  int st = 0;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (st) return set_error(ctx, RMGTD_EDIVERGED, "ground state: the block lost rank (Cholesky pivot)");
  ctx->gs_iters = std::min(it, maxit);
  ctx->gs_err = err;
  ctx->gs_resid = rmax;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(theta.data(), w.theta, sizeof(double) * nt, cudaMemcpyDeviceToHost,
                                  ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->gs_eps.assign(theta.begin(), theta.begin() + N);
  if (!done)
    return set_error(ctx, RMGTD_ENOTCONVERGED,
                     "ground state: " + std::to_string(maxit) + " SCF iterations, max|drho| " +
                         std::to_string(err) + ", residual " + std::to_string(rmax));
  // the N lowest Ritz vectors become the active space (orthonormal, ascending energies)
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->phi, w.X, sizeof(double) * N * Ng, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

}  // namespace rmgtd
