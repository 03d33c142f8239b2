// Propagation variants of Section 2.2 and the spectrum of Section 4:
//  * the non-orthogonal basis: the commutator series with S^-1 Hbar (Appendix A.2 derives it
//    from the orthogonal one through S = L L^T), started from P_0 = L^-T diag(f) L^-1;
//  * the second-order Magnus term Omega_2 = (dt^2/12)[H_0, H_1] for H linear over the step;
//  * the dipole strength function from the kicked dipole series (rmgtd_spectrum).
// The N x N products here are small float64 contractions (at most a few per SCF pass, N <= a
// few hundred), done with 16 x 16 shared-memory tiles.
#include "rmgtd_internal.cuh"

namespace rmgtd {

namespace {

constexpr int kT = 16;   // tile edge of the small float64 products

// X = L^-1 for the lower Cholesky factor L (row-major, upper part ignored): thread j solves
// L x = e_j by forward substitution, x_i = 0 above the diagonal.
__global__ void k_tri_inverse(int N, const double* __restrict__ L, double* __restrict__ X) {
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    for (int i = 0; i < j; ++i) X[(long)i * N + j] = 0.0;
    X[(long)j * N + j] = 1.0 / L[(long)j * N + j];
    for (int i = j + 1; i < N; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s = fma(L[(long)i * N + k], X[(long)k * N + j], s);
      X[(long)i * N + j] = -s / L[(long)i * N + i];
    }
  }
}

// out_r = X^T diag(f) X (f NULL: X^T X) for nrep copies of stride N*N; im (may be NULL) is
// zeroed alongside
__global__ void k_xtdx(int N, int nrep, const double* __restrict__ X, const double* __restrict__ f,
                       double* __restrict__ out, double* __restrict__ im) {
  const long NN = (long)N * N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < NN;
       e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / N), j = (int)(e % N);
    double s = 0.0;
    for (int k = 0; k < N; ++k) {
      const double w = f ? f[k] : 1.0;
      s = fma(X[(long)k * N + i] * w, X[(long)k * N + j], s);
    }
    for (int r = 0; r < nrep; ++r) {
      out[r * NN + e] = s;
      if (im) im[r * NN + e] = 0.0;
    }
  }
}

// C_r = alpha A_r B_r + beta A2_r B2_r (A2 NULL: first product only); operand strides per
// replica may be 0 (shared).  One 16 x 16 output tile per block, one output per thread.
__global__ void __launch_bounds__(kT * kT) k_dgemm_pair(int N, double alpha, const double* __restrict__ A,
                                                        long sa, const double* __restrict__ B, long sb,
                                                        double beta, const double* __restrict__ A2,
                                                        long sa2, const double* __restrict__ B2,
                                                        long sb2, double* __restrict__ C, long sc) {
  __shared__ double tA[kT][kT + 1], tB[kT][kT + 1];
  const int r = blockIdx.z;
  const int ty = threadIdx.x / kT, tx = threadIdx.x % kT;
  const int i = blockIdx.y * kT + ty, j = blockIdx.x * kT + tx;
  double acc[2] = {0.0, 0.0};
  for (int p = 0; p < (A2 ? 2 : 1); ++p) {
    const double* a = (p == 0 ? A + r * sa : A2 + r * sa2);
    const double* b = (p == 0 ? B + r * sb : B2 + r * sb2);
    for (int k0 = 0; k0 < N; k0 += kT) {
      const int ka = k0 + tx, kb = k0 + ty;
      tA[ty][tx] = (i < N && ka < N) ? a[(long)i * N + ka] : 0.0;
      tB[ty][tx] = (kb < N && j < N) ? b[(long)kb * N + j] : 0.0;
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kT; ++k) acc[p] = fma(tA[ty][k], tB[k][tx], acc[p]);
      __syncthreads();
    }
  }
  if (i < N && j < N) C[r * sc + (long)i * N + j] = alpha * acc[0] + (A2 ? beta * acc[1] : 0.0);
}

// mode 0: o1_r = (H0_r + H1_r)/2 + sum_q ebar_rq M_q; mode 1: o1_r = H0_r + sum_q E_rq(t) M_q,
// o2_r = H1_r + sum_q E_rq(t + dt) M_q.  e: the step's field block ([nrep][3] means, then
// [nrep][6] end values) or NULL.
__global__ void k_hx_form(int N, int nrep, const double* __restrict__ H0, const double* __restrict__ H1,
                          long hstride, const double* __restrict__ M, const double* __restrict__ e,
                          int mode, double* __restrict__ o1, double* __restrict__ o2) {
  const long NN = (long)N * N;
  for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < NN * nrep;
       x += (long)gridDim.x * blockDim.x) {
    const int r = (int)(x / NN);
    const long o = x - r * NN;
    const double h0 = H0[r * hstride + o], h1 = H1[r * hstride + o];
    const double m0 = M[o], m1 = M[NN + o], m2 = M[2 * NN + o];
    if (mode == 0) {
      double v = 0.5 * (h0 + h1);
      if (e) v += e[3 * r] * m0 + e[3 * r + 1] * m1 + e[3 * r + 2] * m2;
      o1[x] = v;
    } else {
      double v0 = h0, v1 = h1;
      if (e) {
        const double* ee = e + 3 * nrep + 6 * r;
        v0 += ee[0] * m0 + ee[1] * m1 + ee[2] * m2;
        v1 += ee[3] * m0 + ee[4] * m1 + ee[5] * m2;
      }
      o1[x] = v0;
      o2[x] = v1;
    }
  }
}

int launch_pair(rmgtd_ctx* ctx, int nrep, double alpha, const double* A, long sa, const double* B,
                long sb, double beta, const double* A2, long sa2, const double* B2, long sb2,
                double* C, long sc) {
  const int N = ctx->N;
  const dim3 grid((unsigned)ceil_div(N, kT), (unsigned)ceil_div(N, kT), (unsigned)nrep);
  k_dgemm_pair<<<grid, kT * kT, 0, ctx->stream>>>(N, alpha, A, sa, B, sb, beta, A2, sa2, B2, sb2,
                                                  C, sc);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_dgemm_pair");
  return RMGTD_OK;
}

int elementwise_blocks(rmgtd_ctx* ctx, long n) {
  return (int)std::max<long>(1, std::min<long>(ceil_div(n, 256), 4L * ctx->num_sms));
}

// strength function: g_n = (1/nq) sum_q (d_q(t_n) - d_q(0)) w_n dt e^{-gamma t_n} (w_n: the
// trapezoid weights), then S(omega) = -(2 omega / (pi kappa)) sum_n g_n sin(omega t_n)
__global__ void k_spectrum_signal(int nq, long nt, const double* __restrict__ d, double dt,
                                  double gamma, double* __restrict__ g) {
  for (long n = blockIdx.x * (long)blockDim.x + threadIdx.x; n < nt;
       n += (long)gridDim.x * blockDim.x) {
    const double t = dt * (double)n;
    const double w = (nt == 1) ? 0.0 : ((n == 0 || n == nt - 1) ? 0.5 : 1.0);
    double s = 0.0;
    for (int q = 0; q < nq; ++q) s += d[q * nt + n] - d[q * nt];
    g[n] = s / nq * w * dt * exp(-gamma * t);
  }
}

// one warp per frequency; lanes take every 32nd sample, then a fixed-order warp sum
__global__ void k_spectrum(long nt, const double* __restrict__ g, double dt, double kappa,
                           const double* __restrict__ omega, int nw, double* __restrict__ S) {
  const int lane = threadIdx.x & 31;
  const long wi = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  if (wi >= nw) return;
  const double om = omega[wi];
  double s = 0.0;
  for (long n = lane; n < nt; n += 32) s = fma(g[n], sin(om * (dt * (double)n)), s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) S[wi] = -2.0 * om / (M_PI * kappa) * s;
}

}  // namespace

int nonorth_setup(rmgtd_ctx* ctx) {
  const int N = ctx->N;
  const long NN = (long)N * N;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Hx0, ctx->Smat, sizeof(double) * NN, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  k_cholesky<<<1, 1024, 0, ctx->stream>>>(N, ctx->Hx0, ctx->status);   // L (lower) of S
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_cholesky");
  k_tri_inverse<<<1, 1024, 0, ctx->stream>>>(N, ctx->Hx0, ctx->Hx1);   // X = L^-1
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_tri_inverse");
  const int blocks = elementwise_blocks(ctx, NN);
  k_xtdx<<<blocks, 256, 0, ctx->stream>>>(N, 1, ctx->Hx1, nullptr, ctx->Sinv, nullptr);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_xtdx");
  k_xtdx<<<blocks, 256, 0, ctx->stream>>>(N, ctx->nrep, ctx->Hx1, ctx->f_dev, ctx->S0, ctx->A0);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_xtdx");
  int st = 0;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(&st, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (st) return set_error(ctx, RMGTD_EINVAL, "overlap matrix of phi0 is not positive definite");
  return RMGTD_OK;
}

int magnus_prepare(rmgtd_ctx* ctx, const double** Ha, const double** Hb, long* hstride,
                   const double** febar, const double** D) {
  const int N = ctx->N, nrep = ctx->nrep;
  const long NN = (long)N * N;
  const double* e = ctx->fld_on ? ctx->fld_ebar : nullptr;
  *Ha = ctx->H0;
  *Hb = ctx->H1;
  *hstride = NN;
  *febar = e;
  *D = nullptr;
  const int blocks = elementwise_blocks(ctx, NN * nrep);
  if (ctx->opt.nonorthogonal) {
    k_hx_form<<<blocks, 256, 0, ctx->stream>>>(N, nrep, ctx->H0, ctx->H1, NN, ctx->M, e, 0,
                                               ctx->Hx0, nullptr);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_hx_form");
    int rc = launch_pair(ctx, nrep, 1.0, ctx->Sinv, 0, ctx->Hx0, NN, 0.0, nullptr, 0, nullptr, 0,
                         ctx->Gm, NN);
    if (rc) return rc;
    *Ha = *Hb = ctx->Gm;
    *febar = nullptr;
  }
  if (ctx->opt.magnus_order == 2) {
    const double* A = ctx->H0;
    const double* B = ctx->H1;
    if (e) {
      k_hx_form<<<blocks, 256, 0, ctx->stream>>>(N, nrep, ctx->H0, ctx->H1, NN, ctx->M, e, 1,
                                                 ctx->Hx0, ctx->Hx1);
      ++ctx->launches;
      RMGTD_LAUNCH(ctx, "k_hx_form");
      A = ctx->Hx0;
      B = ctx->Hx1;
    }
    const double c = ctx->opt.dt / 12.0;   // Omega_2 = dt D with D = (dt/12)[A, B]
    int rc = launch_pair(ctx, nrep, c, A, NN, B, NN, -c, B, NN, A, NN, ctx->Dm, NN);
    if (rc) return rc;
    *D = ctx->Dm;
  }
  return RMGTD_OK;
}

int hbar_with_field(rmgtd_ctx* ctx, const double* Ha, const double* Hb, long hstride,
                    const double* febar, int rep0, int nreps, double* out) {
  const int N = ctx->N;
  const long NN = (long)N * N;
  k_hx_form<<<elementwise_blocks(ctx, NN * nreps), 256, 0, ctx->stream>>>(
      N, nreps, Ha, Hb, hstride, ctx->M, febar + 3 * rep0, 0, out, nullptr);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_hx_form");
  return RMGTD_OK;
}

int nonorth_kick_matrix(rmgtd_ctx* ctx, int axis) {
  const long NN = (long)ctx->N * ctx->N;
  return launch_pair(ctx, 1, 1.0, ctx->Sinv, 0, ctx->M + axis * NN, 0, 0.0, nullptr, 0, nullptr, 0,
                     ctx->Gm, 0);
}

}  // namespace rmgtd

using namespace rmgtd;

extern "C" int rmgtd_spectrum(const double* dipole, int nq, long nt, double dt, double kappa,
                              double gamma, const double* omega, int nw, double* S) {
  if (!dipole || !omega || !S || nq < 1 || nq > 64 || nt < 1 || nw < 1 || nw > (1 << 24) ||
      !(dt > 0.0) || !(kappa != 0.0) || !(gamma >= 0.0) || nt > (1L << 36) / nq)
    return set_error(nullptr, RMGTD_EINVAL, "spectrum: bad pointer or size");
  double* dd = nullptr;
  double* g = nullptr;
  double* om = nullptr;
  double* out = nullptr;
  int rc = RMGTD_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && rc == RMGTD_OK) {
      set_error(nullptr, RMGTD_ECUDA, std::string("spectrum: ") + what + ": " + cudaGetErrorString(e));
      rc = RMGTD_ECUDA;
    }
  };
  fail(cudaMalloc(&dd, sizeof(double) * nq * nt), "cudaMalloc");
  if (!rc) fail(cudaMalloc(&g, sizeof(double) * nt), "cudaMalloc");
  if (!rc) fail(cudaMalloc(&om, sizeof(double) * nw), "cudaMalloc");
  if (!rc) fail(cudaMalloc(&out, sizeof(double) * nw), "cudaMalloc");
  if (!rc) fail(cudaMemcpy(dd, dipole, sizeof(double) * nq * nt, cudaMemcpyHostToDevice), "copy in");
  if (!rc) fail(cudaMemcpy(om, omega, sizeof(double) * nw, cudaMemcpyHostToDevice), "copy in");
  if (!rc) {
    const int blocks = (int)std::min<long>((nt + 255) / 256, 4096);
    k_spectrum_signal<<<blocks, 256>>>(nq, nt, dd, dt, gamma, g);
    fail(cudaGetLastError(), "k_spectrum_signal");
  }
  if (!rc) {
    const long threads = 32L * nw;   // <= 2^29
    k_spectrum<<<(unsigned)((threads + 255) / 256), 256>>>(nt, g, dt, kappa, om, nw, out);
    fail(cudaGetLastError(), "k_spectrum");
  }
  if (!rc) fail(cudaMemcpy(S, out, sizeof(double) * nw, cudaMemcpyDeviceToHost), "copy out");
  cudaFree(dd);
  cudaFree(g);
  cudaFree(om);
  cudaFree(out);
  return rc;
}
