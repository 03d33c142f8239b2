// Subspace kernels of Algorithm 1: Gram contractions h^3 A^T diag(w) B (H update, H_core,
// dipole and overlap matrices), the density rho = sum_ij Re(P)_ij phi_i phi_j, the
// commutator expansion of exp(Omega) P exp(Omega^dagger) (Eqs. 19, 33, 35), observables and
// the SCF control word.  All float64.
#include <cooperative_groups.h>
#include <math.h>

#include "rmgtd_internal.cuh"
#include "jacobi.cuh"

namespace rmgtd {

// ---------------------------------------------------------------------------------------
// Gram contraction, split over the grid (K = Ng).  Output tile TS x TS per block; block
// (pair, split, rep) accumulates sum_{g in split} A[i][g] w[g] B[j][g] for its tile into
// part[rep][split][i*N+j].  For sym != 0 only tiles with I <= J are formed.
constexpr int kGT = 32;

__device__ __forceinline__ void pair_from_index(int p, int T, int sym, int& I, int& J) {
  if (!sym) {
    I = p / T;
    J = p % T;
    return;
  }
  int i = 0, rem = p;
  while (rem >= T - i) {
    rem -= T - i;
    ++i;
  }
  I = i;
  J = i + rem;
}

__global__ void __launch_bounds__(256)
k_gram_partial(int N, long Ng, const double* __restrict__ A, const double* __restrict__ B,
               const double* __restrict__ w, long wstride, int sym, int T, long chunk,
               double* __restrict__ part, const RepCtl* __restrict__ ctl) {
  const int rep = blockIdx.z;
  if (ctl && !ctl[rep].active) return;
  __shared__ double As[kGT][kGT + 1];
  __shared__ double Bs[kGT][kGT + 1];
  int I, J;
  pair_from_index(blockIdx.x, T, sym, I, J);
  const int split = blockIdx.y, nsplit = gridDim.y;
  const long g_beg = (long)split * chunk;
  const long g_end = min(Ng, g_beg + chunk);
  const double* wr = w ? w + rep * wstride : nullptr;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc00 = 0, acc01 = 0, acc10 = 0, acc11 = 0;
  for (long g0 = g_beg; g0 < g_end; g0 += kGT) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + 256 * e;
      const int r = idx >> 5, c = idx & 31;
      const long g = g0 + c;
      const int ia = I * kGT + r, jb = J * kGT + r;
      double av = 0.0, bv = 0.0;
      if (g < g_end) {
        if (ia < N) av = A[(long)ia * Ng + g];
        if (jb < N) {
          bv = B[(long)jb * Ng + g];
          if (wr) bv *= wr[g];
        }
      }
      As[c][r] = av;
      Bs[c][r] = bv;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kGT; ++k) {
      const double a0 = As[k][ty], a1 = As[k][ty + 16];
      const double b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
      acc00 = fma(a0, b0, acc00);
      acc01 = fma(a0, b1, acc01);
      acc10 = fma(a1, b0, acc10);
      acc11 = fma(a1, b1, acc11);
    }
    __syncthreads();
  }
  // element-major partials [rep][i*N+j][split]: the reduction reads them contiguously
  double* out = part + (long)rep * N * N * nsplit + split;
  const int i0 = I * kGT + ty, i1 = i0 + 16, j0 = J * kGT + tx, j1 = j0 + 16;
  if (i0 < N && j0 < N) out[((long)i0 * N + j0) * nsplit] = acc00;
  if (i0 < N && j1 < N) out[((long)i0 * N + j1) * nsplit] = acc01;
  if (i1 < N && j0 < N) out[((long)i1 * N + j0) * nsplit] = acc10;
  if (i1 < N && j1 < N) out[((long)i1 * N + j1) * nsplit] = acc11;
}

// out[rep] = base + scale * sum_split part; symmetric outputs are mirrored.  One warp per
// output element sums its split partials (contiguous, fixed order).  When `prev` is given,
// max_ij |out - prev| is folded into errbits[rep] (prev may alias out: every element is read
// and written by the same warp).
__global__ void k_gram_reduce(int N, int nsplit, const double* __restrict__ part, double scale,
                              const double* __restrict__ base, long bstride, double* out,
                              long ostride, const double* prev, int sym,
                              unsigned long long* errbits, const RepCtl* __restrict__ ctl) {
  const int rep = blockIdx.y;
  if (ctl && !ctl[rep].active) return;
  __shared__ double sh[32];
  const long NN = (long)N * N;
  const int lane = threadIdx.x & 31;
  const long warps = (long)gridDim.x * (blockDim.x >> 5);
  double emax = 0.0;
  for (long e = blockIdx.x * (long)(blockDim.x >> 5) + (threadIdx.x >> 5); e < NN; e += warps) {
    const int i = (int)(e / N), j = (int)(e % N);
    if (sym && j < i) continue;
    const double* p = part + ((long)rep * NN + e) * nsplit;
    double sacc = 0.0;
    for (int k = lane; k < nsplit; k += 32) sacc += p[k];
    sacc = warp_sum(sacc);
    if (lane == 0) {
      double v = scale * sacc;
      if (base) v += base[rep * bstride + e];
      double* o = out + rep * ostride;
      if (prev) emax = fmax(emax, fabs(v - prev[rep * ostride + e]));
      o[e] = v;
      if (sym && i != j) o[(long)j * N + i] = v;
    }
  }
  if (errbits) {
    emax = block_max(emax, sh);
    if (threadIdx.x == 0) atomic_max_nonneg(&errbits[rep], emax);
  }
}

static int gram_nsplit(rmgtd_ctx* ctx, int ntiles, int nrep) {
  const long target = 4L * ctx->num_sms;
  long ns = (target + (long)ntiles * nrep - 1) / ((long)ntiles * nrep);
  ns = std::max<long>(1, std::min<long>(ns, ctx->Ng / 256 + 1));
  // partial buffer bound
  const long per = (long)nrep * ctx->N * ctx->N;
  ns = std::min<long>(ns, (long)(ctx->gram_part_elems / std::max<long>(per, 1)));
  return (int)std::max<long>(ns, 1);
}

int gram(rmgtd_ctx* ctx, const double* A, const double* B, const double* w, long wstride,
         int nw, double scale, const double* base, double* out, const double* prev,
         const RepCtl* ctl, int sym, unsigned long long* errbits, long bstride) {
  const int N = ctx->N;
  const int T = ceil_div(N, kGT);
  const int ntiles = sym ? T * (T + 1) / 2 : T * T;
  const int nsplit = gram_nsplit(ctx, ntiles, nw);
  const long chunk = ((ctx->Ng + nsplit - 1) / nsplit + kGT - 1) / kGT * kGT;
  dim3 grid(ntiles, nsplit, nw);
  k_gram_partial<<<grid, 256, 0, ctx->stream>>>(N, ctx->Ng, A, B, w, wstride, sym, T, chunk,
                                                 ctx->gram_part, ctl);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gram_partial");
  const long NN = (long)N * N;
  const int rb = (int)std::min<long>(ceil_div(NN, 8), 4L * ctx->num_sms);
  k_gram_reduce<<<dim3(rb, nw), 256, 0, ctx->stream>>>(N, nsplit, ctx->gram_part, scale, base,
                                                        bstride, out, NN, prev, sym, errbits, ctl);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gram_reduce");
  return RMGTD_OK;
}

// ---------------------------------------------------------------------------------------
// Density rho(g) = sum_ij S_ij phi_i(g) phi_j(g) with S = Re P symmetric, evaluated as
// sum_j phi_j(g) X_j(g), X_j = sum_{k<=j} Shat_kj phi_k(g), Shat_kj = 2 S_kj (k<j), S_jj
// (k=j): half of the N^2 products.  One thread per grid point, 32 columns j at a time.
constexpr int kRhoJ = 32, kRhoK = 64, kRhoThreads = 128;

__global__ void __launch_bounds__(kRhoThreads)
k_rho(int N, long Ng, const double* __restrict__ phi, const double* __restrict__ S,
      long sstride, double* __restrict__ rho, long rstride, const RepCtl* __restrict__ ctl) {
  const int rep = blockIdx.y;
  if (ctl && !ctl[rep].active) return;
  __shared__ double Sh[kRhoK][kRhoJ];
  const double* Sr = S + rep * sstride;
  const long g = blockIdx.x * (long)kRhoThreads + threadIdx.x;
  const bool ok = g < Ng;
  double r = 0.0;
  for (int jb = 0; jb < N; jb += kRhoJ) {
    double acc[kRhoJ];
#pragma unroll
    for (int jj = 0; jj < kRhoJ; ++jj) acc[jj] = 0.0;
    const int kend = min(N, jb + kRhoJ);
    for (int k0 = 0; k0 < kend; k0 += kRhoK) {
      __syncthreads();
      for (int e = threadIdx.x; e < kRhoK * kRhoJ; e += kRhoThreads) {
        const int kk = e / kRhoJ, jj = e % kRhoJ;
        const int k = k0 + kk, j = jb + jj;
        double v = 0.0;
        if (k < N && j < N) {
          if (k < j)
            v = 2.0 * Sr[(long)k * N + j];
          else if (k == j)
            v = Sr[(long)j * N + j];
        }
        Sh[kk][jj] = v;
      }
      __syncthreads();
      const int kn = min(kRhoK, kend - k0);
      if (ok) {
        for (int kk = 0; kk < kn; ++kk) {
          const double pk = phi[(long)(k0 + kk) * Ng + g];
#pragma unroll
          for (int jj = 0; jj < kRhoJ; ++jj) acc[jj] = fma(Sh[kk][jj], pk, acc[jj]);
        }
      }
    }
    if (ok) {
#pragma unroll
      for (int jj = 0; jj < kRhoJ; ++jj)
        if (jb + jj < N) r = fma(phi[(long)(jb + jj) * Ng + g], acc[jj], r);
    }
  }
  if (ok) rho[rep * rstride + g] = r;
}

int rho_dev(rmgtd_ctx* ctx, const double* S, double* rho, const RepCtl* ctl, int nrep) {
  dim3 grid(ceil_div(ctx->Ng, kRhoThreads), nrep);
  k_rho<<<grid, kRhoThreads, 0, ctx->stream>>>(ctx->N, ctx->Ng, ctx->phi, S,
                                                (long)ctx->N * ctx->N, rho, ctx->Ng, ctl);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_rho");
  return RMGTD_OK;
}

// ---------------------------------------------------------------------------------------
// Mixed-precision contractions around the float64 reference state (P_ref, V_ref):
//   rho = rho_ref + sum_ij (S - S_ref)_ij phi_i phi_j      (float32 products and sums)
//   H   = H_ref + h^3 Phi^T diag(V - V_ref) Phi            (float32 per block, float64 across)
// Rounding then scales with the perturbation P - P_ref, not with P.
// Density of the change of P: the float32 matrix Shat_kj = 2 dS_kj (k < j), dS_jj (k = j),
// 0 (k > j), dS = S - S_ref, zero-padded to Np x Np (Np = N rounded up to 32), formed once
// per pass by k_shat32 and streamed by k_rho32.
__global__ void k_shat32(int N, int Np, const double* __restrict__ S, const double* __restrict__ Sref,
                         long sstride, float* __restrict__ shat, const RepCtl* __restrict__ ctl) {
  const int rep = blockIdx.y;
  if (ctl && !ctl[rep].active) return;
  const double* Sr = S + rep * sstride;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < (long)Np * Np;
       e += (long)gridDim.x * blockDim.x) {
    const int k = (int)(e / Np), j = (int)(e % Np);
    double v = 0.0;
    if (k < N && j < N && k <= j) {
      const long o = (long)k * N + j;
      v = (k < j) ? 2.0 * (Sr[o] - Sref[o]) : (Sr[o] - Sref[o]);
    }
    shat[(long)rep * Np * Np + e] = (float)v;
  }
}

// rho = rho_ref + drho, drho = sum_j phi_j X_j (also stored in float32 for the Hartree
// solve), X_j = sum_{k<=j} Shat_kj phi_k: each thread two grid
// points (g, g + 128), 32 columns j at a time, Shat rows read as float4 broadcasts.
constexpr int kRho32Pts = 2;
__global__ void __launch_bounds__(kRhoThreads)
k_rho32(int N, int Np, long Ng, const float* __restrict__ phi, const float* __restrict__ shat,
        const double* __restrict__ rho_ref, double* __restrict__ rho, float* __restrict__ drho,
        long rstride, const RepCtl* __restrict__ ctl) {
  const int rep = blockIdx.y;
  if (ctl && !ctl[rep].active) return;
  __shared__ __align__(16) float Sh[kRhoK][kRhoJ];
  const float* shr = shat + (long)rep * Np * Np;
  const long g0 = blockIdx.x * (long)(kRhoThreads * kRho32Pts) + threadIdx.x;
  const long g1 = g0 + kRhoThreads;
  const bool ok0 = g0 < Ng, ok1 = g1 < Ng;
  float r0 = 0.0f, r1 = 0.0f;
  for (int jb = 0; jb < N; jb += kRhoJ) {
    float a0[kRhoJ], a1[kRhoJ];
#pragma unroll
    for (int jj = 0; jj < kRhoJ; ++jj) a0[jj] = a1[jj] = 0.0f;
    const int kend = min(N, jb + kRhoJ);
    for (int k0 = 0; k0 < kend; k0 += kRhoK) {
      __syncthreads();
      // stage Shat[k0 .. k0+63][jb .. jb+31] (float4, coalesced; padded rows are zero)
      for (int e = threadIdx.x; e < kRhoK * kRhoJ / 4; e += kRhoThreads) {
        const int kk = e / (kRhoJ / 4), q = e % (kRhoJ / 4);
        const int k = k0 + kk;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < Np) v = *reinterpret_cast<const float4*>(shr + (long)k * Np + jb + 4 * q);
        *reinterpret_cast<float4*>(&Sh[kk][4 * q]) = v;
      }
      __syncthreads();
      const int kn = min(kRhoK, kend - k0);
      int kk = 0;
      for (; kk + 1 < kn; kk += 2) {
        const long ka = (long)(k0 + kk) * Ng, kb = ka + Ng;
        const float pa0 = ok0 ? phi[ka + g0] : 0.f, pa1 = ok1 ? phi[ka + g1] : 0.f;
        const float pb0 = ok0 ? phi[kb + g0] : 0.f, pb1 = ok1 ? phi[kb + g1] : 0.f;
        const float4* ra = reinterpret_cast<const float4*>(&Sh[kk][0]);
        const float4* rb = reinterpret_cast<const float4*>(&Sh[kk + 1][0]);
#pragma unroll
        for (int q = 0; q < kRhoJ / 4; ++q) {
          const float4 u = ra[q], w = rb[q];
          a0[4 * q + 0] = fmaf(w.x, pb0, fmaf(u.x, pa0, a0[4 * q + 0]));
          a0[4 * q + 1] = fmaf(w.y, pb0, fmaf(u.y, pa0, a0[4 * q + 1]));
          a0[4 * q + 2] = fmaf(w.z, pb0, fmaf(u.z, pa0, a0[4 * q + 2]));
          a0[4 * q + 3] = fmaf(w.w, pb0, fmaf(u.w, pa0, a0[4 * q + 3]));
          a1[4 * q + 0] = fmaf(w.x, pb1, fmaf(u.x, pa1, a1[4 * q + 0]));
          a1[4 * q + 1] = fmaf(w.y, pb1, fmaf(u.y, pa1, a1[4 * q + 1]));
          a1[4 * q + 2] = fmaf(w.z, pb1, fmaf(u.z, pa1, a1[4 * q + 2]));
          a1[4 * q + 3] = fmaf(w.w, pb1, fmaf(u.w, pa1, a1[4 * q + 3]));
        }
      }
      if (kk < kn) {
        const long ka = (long)(k0 + kk) * Ng;
        const float pa0 = ok0 ? phi[ka + g0] : 0.f, pa1 = ok1 ? phi[ka + g1] : 0.f;
        const float4* ra = reinterpret_cast<const float4*>(&Sh[kk][0]);
#pragma unroll
        for (int q = 0; q < kRhoJ / 4; ++q) {
          const float4 u = ra[q];
          a0[4 * q + 0] = fmaf(u.x, pa0, a0[4 * q + 0]);
          a0[4 * q + 1] = fmaf(u.y, pa0, a0[4 * q + 1]);
          a0[4 * q + 2] = fmaf(u.z, pa0, a0[4 * q + 2]);
          a0[4 * q + 3] = fmaf(u.w, pa0, a0[4 * q + 3]);
          a1[4 * q + 0] = fmaf(u.x, pa1, a1[4 * q + 0]);
          a1[4 * q + 1] = fmaf(u.y, pa1, a1[4 * q + 1]);
          a1[4 * q + 2] = fmaf(u.z, pa1, a1[4 * q + 2]);
          a1[4 * q + 3] = fmaf(u.w, pa1, a1[4 * q + 3]);
        }
      }
    }
#pragma unroll
    for (int jj = 0; jj < kRhoJ; ++jj) {
      if (jb + jj < N) {
        const long kj = (long)(jb + jj) * Ng;
        if (ok0) r0 = fmaf(phi[kj + g0], a0[jj], r0);
        if (ok1) r1 = fmaf(phi[kj + g1], a1[jj], r1);
      }
    }
  }
  if (ok0) {
    if (rho) rho[rep * rstride + g0] = rho_ref[g0] + (double)r0;
    drho[rep * rstride + g0] = r0;
  }
  if (ok1) {
    if (rho) rho[rep * rstride + g1] = rho_ref[g1] + (double)r1;
    drho[rep * rstride + g1] = r1;
  }
}

int rho_dev_mixed(rmgtd_ctx* ctx, const double* S, double* rho, const RepCtl* ctl, int nrep) {
  const int N = ctx->N, Np = ((N + 31) / 32) * 32;
  const long NpNp = (long)Np * Np;
  if (ctx->phi_pl) {   // orbital planes on the tensor cores (32 < N <= 256)
    ctx->shat_fresh = 0;
    return rho_planes(ctx, S, rho, ctx->drho32, ctl, nrep);
  }
  if (!ctx->shat_fresh || S != ctx->S1) {
    k_shat32<<<dim3(std::max(1, (int)std::min<long>(ceil_div(NpNp, 256), 1024)), nrep), 256, 0,
               ctx->stream>>>(N, Np, S, ctx->Sref, (long)N * N, ctx->shat32, ctl);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_shat32");
  }
  ctx->shat_fresh = 0;
  const int rc = rho_tc(ctx, rho, ctx->drho32, ctl, nrep);   // tensor cores when N <= 32
  if (rc <= 0) return rc;
  dim3 grid(ceil_div(ctx->Ng, kRhoThreads * kRho32Pts), nrep);
  k_rho32<<<grid, kRhoThreads, 0, ctx->stream>>>(N, Np, ctx->Ng, ctx->phi32, ctx->shat32,
                                                  ctx->rho_ref, rho, ctx->drho32, ctx->Ng, ctl);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_rho32");
  return RMGTD_OK;
}

// float32 H update of the mixed path: C_r = sum_g phi_i(g) w_r(g) phi_j(g) for every replica
// r, i <= j.  Block = 4 k-groups x 128 threads; each k-group takes 32 of the 128 grid points
// staged per slab.  A thread owns one 4 x 4 sub-tile of the 32 x 32 output tile pair
// (It, Jt) for one replica: in a diagonal tile pair only the 36 sub-tiles on or above the
// diagonal are formed (3 replicas per block), otherwise all 64 (2 replicas per block).  The
// staged orbital slab serves every replica of the block.  The 4 k-groups are summed in
// shared memory and each block writes its float32 partial tile [split][rep][Np][Np].
constexpr int kG32Slab = 128;               // grid points staged per slab
constexpr int kG32Groups = 4;               // k-groups per block
constexpr int kG32Group = 128;              // threads per k-group
constexpr int kG32Threads = kG32Groups * kG32Group;
constexpr int kG32Pad = kGT + 4;   // 144-byte rows: float4 reads, conflict-free staging

struct Gram32Smem {
  union {
    struct {
      float A[kG32Slab][kG32Pad];   // [k][i] rows of tile It
      float B[kG32Slab][kG32Pad];   // [k][j] rows of tile Jt
      float W[kG32Slab][4];         // [k][replica of the block]
    } s;
    float red[kG32Groups - 1][kG32Group][16];
  };
};

// sub-tile (I4, J4) of item s: diagonal pair -> upper-triangle enumeration of the 8 x 8 grid
__device__ __forceinline__ void subtile_of(int s, bool diag, int& I4, int& J4) {
  if (!diag) {
    I4 = s >> 3;
    J4 = s & 7;
    return;
  }
  int i = 0, rem = s;
  while (rem >= 8 - i) {
    rem -= 8 - i;
    ++i;
  }
  I4 = i;
  J4 = i + rem;
}

__global__ void __launch_bounds__(kG32Threads)
k_gram32(int N, int Np, int Ng, const float* __restrict__ phi, const float* __restrict__ w,
         int nrep, int T, int chunk, float* __restrict__ part, const RepCtl* __restrict__ ctl) {
  __shared__ __align__(16) Gram32Smem sm;
  int It, Jt;
  pair_from_index(blockIdx.y, T, 1, It, Jt);
  const bool diag = (It == Jt);
  const int per_rep = diag ? 36 : 64;
  const int R = diag ? 3 : 2;                  // replicas per block
  const int rep0 = blockIdx.z * R;
  if (rep0 >= nrep) return;
  const int nr = min(R, nrep - rep0);
  const int split = blockIdx.x;
  const int g_beg = split * chunk;
  const int g_end = min(Ng, g_beg + chunk);
  const int tid = threadIdx.x, kg = tid / kG32Group, u = tid % kG32Group;
  const bool work = u < nr * per_rep;
  const int rl = work ? u % nr : 0;           // replica (minor) and sub-tile (major)
  int I4 = 0, J4 = 0;
  if (work) subtile_of(u / nr, diag, I4, J4);
  const bool rep_on = work && (!ctl || ctl[rep0 + rl].active);
  float acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0f;
  for (int g0 = g_beg; g0 < g_end; g0 += kG32Slab) {
    __syncthreads();
    // stage: lane <-> orbital row (conflict-free transposed stores), 4 points per load
    for (int e = tid; e < 2 * kGT * (kG32Slab / 4); e += kG32Threads) {
      const int which = e / (kGT * (kG32Slab / 4));     // 0: tile It, 1: tile Jt
      const int r = e % kGT, q = (e / kGT) % (kG32Slab / 4);
      if (which == 1 && diag) continue;
      const int row = (which ? Jt : It) * kGT + r;
      const int g = g0 + 4 * q;
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      if (row < N) {
        const float* src = phi + (long)row * Ng + g;
        if (g + 3 < g_end && ((((long)row * Ng + g) & 3) == 0)) {
          const float4 t = *reinterpret_cast<const float4*>(src);
          v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (g + c < g_end) v[c] = src[c];
        }
      }
      float(*dst)[kG32Pad] = which ? sm.s.B : sm.s.A;
#pragma unroll
      for (int c = 0; c < 4; ++c) dst[4 * q + c][r] = v[c];
    }
    for (int e = tid; e < kG32Slab * 4; e += kG32Threads) {
      const int k = e >> 2, rr = e & 3;
      const int g = g0 + k;
      sm.s.W[k][rr] = (rr < nr && g < g_end) ? w[(long)(rep0 + rr) * Ng + g] : 0.0f;
    }
    __syncthreads();
    if (rep_on) {
      const float(*Bt)[kG32Pad] = diag ? sm.s.A : sm.s.B;
#pragma unroll 4
      for (int kk = 0; kk < kG32Slab / kG32Groups; ++kk) {
        const int k = kg * (kG32Slab / kG32Groups) + kk;
        const float4 a = *reinterpret_cast<const float4*>(&sm.s.A[k][4 * I4]);
        const float4 b = *reinterpret_cast<const float4*>(&Bt[k][4 * J4]);
        const float wv = sm.s.W[k][rl];
        const float av[4] = {a.x, a.y, a.z, a.w};
        const float bv[4] = {b.x * wv, b.y * wv, b.z * wv, b.w * wv};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(av[p], bv[q], acc[p][q]);
      }
    }
  }
  // sum the k-groups (fixed order), then write this block's partial tile
  __syncthreads();
  if (kg > 0) {
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) sm.red[kg - 1][u][4 * p + q] = acc[p][q];
  }
  __syncthreads();
  if (kg == 0 && work) {
    const long NpNp = (long)Np * Np;
    float* out = part + ((long)split * nrep + rep0 + rl) * NpNp;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int i = It * kGT + 4 * I4 + p;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float v = acc[p][q];
        for (int g = 0; g < kG32Groups - 1; ++g) v += sm.red[g][u][4 * p + q];
        out[(long)i * Np + Jt * kGT + 4 * J4 + q] = rep_on ? v : 0.0f;
      }
    }
  }
}

// out[rep] = base + scale * sum_split part (fixed order), mirrored to i > j;
// max_ij |out - prev| folded into errbits.  Block = 32 warps x 32 consecutive elements of
// one replica; warp w sums the splits s = w, w + 32, ... (8 loads in flight per lane), so a
// few hundred splits take one or two rounds of L2 latency.
__global__ void __launch_bounds__(1024)
k_gram32_reduce(int N, int Np, int nsplit, int nrep, const float* __restrict__ part,
                double scale, const double* __restrict__ base, long bstride, double* out,
                const double* prev, unsigned long long* errbits, const RepCtl* __restrict__ ctl) {
  const int rep = blockIdx.y;
  if (ctl && !ctl[rep].active) return;
  __shared__ double sh[32][33];
  const long NpNp = (long)Np * Np;
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const long e = (long)blockIdx.x * 32 + lane;
  // Eight independent loads in flight per step, summed in split order as an unevaluated
  // float pair (hi + lo, Knuth's two-sum: the rounding error of every addition is kept), so
  // the sum carries ~2^-44 relative error with float32 instructions only -- GB300's float64
  // rate (~1/64) made the former float64 accumulation the kernel's bound.
  float shi = 0.0f, slo = 0.0f;
  // only the upper triangle i <= j is used (mirrored below)
  if (e < NpNp && (int)(e % Np) >= (int)(e / Np)) {
    for (int k0 = wp; k0 < nsplit; k0 += 256) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + 32 * u;
        v[u] = k < nsplit ? part[((long)k * nrep + rep) * NpNp + e] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float t = shi + v[u];
        const float bp = t - shi;
        slo += (shi - (t - bp)) + (v[u] - bp);
        shi = t;
      }
    }
  }
  const double s = (double)shi + (double)slo;
  sh[wp][lane] = s;
  __syncthreads();
  double emax = 0.0;
  if (wp == 0 && e < NpNp) {
    double t = 0.0;
    for (int k = 0; k < 32; ++k) t += sh[k][lane];
    const int i = (int)(e / Np), j = (int)(e % Np);
    if (i < N && j < N && i <= j) {
      const long NN = (long)N * N;
      const long o = (long)i * N + j;
      double v = scale * t;
      if (base) v += base[rep * bstride + o];
      double* orow = out + rep * NN;
      if (prev) emax = fmax(emax, fabs(v - prev[rep * NN + o]));
      orow[o] = v;
      if (i != j) orow[(long)j * N + i] = v;
    }
  }
  if (errbits) {
    if (wp == 0) {
      emax = warp_max(emax);
      if (lane == 0) atomic_max_nonneg(&errbits[rep], emax);
    }
  }
}

int gram_mixed(rmgtd_ctx* ctx, const float* w, long wstride, int nw, double scale,
               const double* base, double* out, const RepCtl* ctl, unsigned long long* errbits,
               long bstride, const float* w_anchor) {
  const int N = ctx->N;
  const int T = ceil_div(N, kGT);
  const int Np = T * kGT;
  const int npairs = T * (T + 1) / 2;
  if (wstride != ctx->Ng) return set_error(ctx, RMGTD_EINVAL, "gram_mixed: replica stride must be Ng");
  const int ngroups = ceil_div(nw, 2);   // replica groups of off-diagonal pairs (diagonal: 3)
  // tune_gram_blocks CTAs per SM over the (pair, replica-group) units: groups of 4 replicas
  // on the tensor cores, of 3 (diagonal pairs) in the SIMT kernel; bounded by the partials
  const bool tc = ctx->tune_gram_tc != 0;
  long ns = ceil_div((long)std::max(1, ctx->tune_gram_blocks) * ctx->num_sms,
                     (long)npairs * ceil_div(nw, tc ? 4 : 3));
  ns = std::max<long>(1, std::min<long>(ns, ceil_div(ctx->Ng, (long)kG32Slab)));
  const long per = (long)nw * Np * Np;   // floats per split
  ns = std::min<long>(ns, (long)(2 * ctx->gram_part_elems) / std::max<long>(per, 1));
  if (ns < 1) return set_error(ctx, RMGTD_ENOMEM, "gram_mixed: partial buffer too small");
  int nsplit = (int)ns;
  int chunk = (int)(ceil_div(ceil_div(ctx->Ng, (long)nsplit), (long)kG32Slab) * kG32Slab);
  nsplit = (int)ceil_div(ctx->Ng, (long)chunk);   // no empty splits
  float* part = reinterpret_cast<float*>(ctx->gram_part);
  int rc = 1;
  // anchored weights exist only with the orbital planes, whose Gram is then always used (a
  // tuning choice of the other Gram kernels applies to contexts without planes)
  if ((tc || w_anchor) && ctx->phi_pl) {
    // orbital planes: one CTA per SM over (split, replica), chunks of whole 64-point stages
    int ps = std::max(1, ctx->num_sms / nw);
    ps = (int)std::min<long>(ps, (long)(2 * ctx->gram_part_elems) / std::max<long>(per, 1));
    const int pchunk = (int)(ceil_div(ceil_div(ctx->Ng, (long)ps), 64L) * 64);
    const int pns = (int)ceil_div(ctx->Ng, (long)pchunk);
    rc = gram_planes(ctx, w, w_anchor, nw, part, pns, pchunk, ctl);
    if (rc == 0) {
      nsplit = pns;
      chunk = pchunk;
    }
  }
  if (w_anchor && rc != 0)
    return rc < 0 ? rc
                  : set_error(ctx, RMGTD_ESTATE,
                              std::string("gram_mixed: anchored weights need the orbital planes (") +
                                  (ctx->phi_pl ? "planes declined" : "no planes") + ", tc " +
                                  std::to_string((int)tc) + ")");
  if (rc > 0 && tc) rc = gram_tc(ctx, w, nw, part, nsplit, chunk, ctl);
  if (rc < 0) return rc;
  if (rc > 0) {
    k_gram32<<<dim3(nsplit, npairs, ngroups), kG32Threads, 0, ctx->stream>>>(
        N, Np, (int)ctx->Ng, ctx->phi32, w, nw, T, chunk, part, ctl);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gram32");
  }
  k_gram32_reduce<<<dim3(ceil_div((long)Np * Np, 32L), nw), 1024, 0, ctx->stream>>>(
      N, Np, nsplit, nw, part, scale, base, bstride, out, out, errbits, ctl);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gram32_reduce");
  return RMGTD_OK;
}

__global__ void k_to_float(long n, const double* __restrict__ in, float* __restrict__ out) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

__global__ void k_tile_orbitals(int N, int Np, long Ng, const float* __restrict__ phi,
                                float* __restrict__ phit, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const long tile = e / (32L * Np);
    const int k = (int)((e >> 5) % Np);
    const long g = tile * 32 + (e & 31);
    phit[e] = (k < N && g < Ng) ? phi[(long)k * Ng + g] : 0.0f;
  }
}

int tile_orbitals(rmgtd_ctx* ctx) {
  const int Np = ((ctx->N + 31) / 32) * 32;
  const long n = ceil_div(ctx->Ng, 32L) * Np * 32;
  const int blocks = (int)std::max<long>(1, std::min<long>(ceil_div(n, 256), 8L * ctx->num_sms));
  k_tile_orbitals<<<blocks, 256, 0, ctx->stream>>>(ctx->N, Np, ctx->Ng, ctx->phi32, ctx->phi32t, n);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_tile_orbitals");
  return RMGTD_OK;
}

__global__ void k_add_fields(long n, const double* __restrict__ a, const double* __restrict__ b,
                             double* __restrict__ out) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x)
    out[e] = a[e] + b[e];
}

int add_fields(rmgtd_ctx* ctx, const double* a, const double* b, double* out, long n) {
  const int blocks = (int)std::max<long>(1, std::min<long>(ceil_div(n, 256), 8L * ctx->num_sms));
  k_add_fields<<<blocks, 256, 0, ctx->stream>>>(n, a, b, out);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_add_fields");
  return RMGTD_OK;
}

int to_float(rmgtd_ctx* ctx, const double* in, float* out, long n) {
  const int blocks = (int)std::max<long>(1, std::min<long>(ceil_div(n, 256), 8L * ctx->num_sms));
  k_to_float<<<blocks, 256, 0, ctx->stream>>>(n, in, out);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_to_float");
  return RMGTD_OK;
}

// ---------------------------------------------------------------------------------------
// Commutator expansion (Algorithm 1's series) in the real split of Eq. 35.  With
// P = S + iA (S symmetric, A antisymmetric), Hbar real symmetric and Omega = -i tau Hbar:
//   S_k =  (tau/k) [Hbar, A_{k-1}] = (tau/k) (T1 + T1^T),  T1 = Hbar A_{k-1}
//   A_k = -(tau/k) [Hbar, S_{k-1}] = -(tau/k) (T2 - T2^T), T2 = Hbar S_{k-1}
// starting from (S_0, A_0) = P_0, P_1 = sum_k (S_k, A_k), stopped when
// max_ij |S_k + i A_k| <= thrs.  One cooperative launch runs the whole series for every
// replica: each block owns symmetric tile pairs (I <= J) and forms T1, T2 for (I,J) and
// (J,I), so the transpose in the commutator never leaves the block; one grid barrier per
// term publishes the new terms and the per-term maxima.
struct EldynArgs {
  int N;
  int nrep;            // replicas in this launch
  int rep0;            // first replica index (for ctl / slots)
  const double* Ha;    // Hbar = (Ha + Hb)/2, replica stride hstride
  const double* Hb;
  long hstride;
  double tau;
  const double* S0;    // [rep][N*N] inputs
  const double* A0;
  double* S1;          // [rep][N*N] outputs
  double* A1;
  double* dbuf;        // [rep][2][2][N*N]
  const RepCtl* ctl_in;   // active flags (NULL: all active)
  RepCtl* ctl_out;        // term statistics (NULL: none)
  unsigned long long* slots;  // [rep][max_terms+1]
  int max_terms;
  double thrs;
  unsigned* bar;
  int* status;
  // optional (cluster kernel): float32 Shat of the new P_1 for the mixed density, rows
  // padded to Np: Shat_kj = 2 (S - Sref)_kj (k < j), (S - Sref)_kk, 0 below the diagonal
  float* shat;
  const double* Sref;
  int Np;
  // external field of the step (NULL: none): Hbar += sum_q ebar[rep][q] M_q, ebar the mean of
  // E(t_j) and E(t_j + dt) (Algorithm 1's V_{j-1} + V_j in Omega)
  const double* fM;       // [3][N*N] dipole matrices
  const double* febar;    // [rep][3]
  // float32 tail (mixed path, cooperative kernel): terms k >= kf from hbar32 = Hbar in float32
  // and the previous term in float32 (dbuf32 [rep][2][2][N*N]); P_1 stays float64.  kf = 0:
  // every term in float64
  int kf;
  const float* hbar32;
  float* dbuf32;
  // second-order Magnus term (NULL: none): Omega = -i tau (Hbar + i D), D = (tau/12)[H_0, H_1]
  // real antisymmetric per replica (stride N*N), so the series multiplies by the Hermitian
  // K = Hbar + i D: T1 = Im(K dP) = Hbar A + D S, T2 = Re(K dP) = Hbar S - D A
  const double* D;
};

// the field's contribution to Hbar at element o of replica rep (0 without a field)
__device__ __forceinline__ double field_term(const EldynArgs& a, int rep, long o) {
  if (!a.febar) return 0.0;
  const long NN = (long)a.N * a.N;
  const double* e = a.febar + 3 * rep;
  return e[0] * a.fM[o] + e[1] * a.fM[NN + o] + e[2] * a.fM[2 * NN + o];
}

template <int TS, int NT, bool WD, bool FT>
__global__ void __launch_bounds__(NT) k_eldyn(EldynArgs a) {
  constexpr int KC = 32;
  constexpr int TSP = TS + 1;
  constexpr int OPT = (4 * TS * TS) / NT;
  static_assert(OPT >= 1 && OPT * NT == 4 * TS * TS, "threads must divide the 4 output tiles");
  extern __shared__ double smem[];
  double* Hi = smem;                 // [TS][KC+1]
  double* Hj = Hi + TS * (KC + 1);
  double* Ai = Hj + TS * (KC + 1);   // [KC][TSP]
  double* Aj = Ai + KC * TSP;
  double* Si = Aj + KC * TSP;
  double* Sj = Si + KC * TSP;
  double* Tt = Sj + KC * TSP;        // [4][TS][TSP]
  double* Di = Tt + 4 * TS * TSP;    // [TS][KC+1] rows of D (only with the Omega_2 term)
  double* Dj = Di + TS * (KC + 1);
  constexpr bool wd = WD;   // with the Omega_2 term (a.D != NULL)
  float* fHi = reinterpret_cast<float*>(Hi);   // float32 views of the tiles (float32 tail)
  float* fHj = reinterpret_cast<float*>(Hj);
  float* fAi = reinterpret_cast<float*>(Ai);
  float* fAj = reinterpret_cast<float*>(Aj);
  float* fSi = reinterpret_cast<float*>(Si);
  float* fSj = reinterpret_cast<float*>(Sj);
  __shared__ double sh[32];
  __shared__ int conv[32];
  __shared__ int all_done;

  const int N = a.N;
  const long NN = (long)N * N;
  const int T = (N + TS - 1) / TS;
  const int npairs = T * (T + 1) / 2;
  const int total = npairs * a.nrep;
  const int tid = threadIdx.x;

  if (tid < 32) {
    int c = 1;
    if (tid < a.nrep) c = (a.ctl_in && !a.ctl_in[a.rep0 + tid].active) ? 1 : 0;
    conv[tid] = c;
  }
  __syncthreads();

  // P_1 <- P_0 on the owned tiles
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int rep = item / npairs;
    if (conv[rep]) continue;
    int I, J;
    pair_from_index(item % npairs, T, 1, I, J);
    for (int e = tid; e < TS * TS; e += NT) {
      const int i = I * TS + e / TS, j = J * TS + e % TS;
      if (i < N && j < N) {
        const long o = rep * NN + (long)i * N + j, ot = rep * NN + (long)j * N + i;
        a.S1[o] = a.S0[o];
        a.A1[o] = a.A0[o];
        if (I != J) {
          a.S1[ot] = a.S0[ot];
          a.A1[ot] = a.A0[ot];
        }
      }
    }
  }

  int k = 0;
  while (true) {
    ++k;
    const double c = a.tau / (double)k;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
      const int rep = item / npairs;
      if (conv[rep]) continue;
      int I, J;
      pair_from_index(item % npairs, T, 1, I, J);
      const double* dS = (k == 1) ? a.S0 + rep * NN : a.dbuf + ((long)rep * 4 + ((k - 1) & 1) * 2) * NN;
      const double* dA = (k == 1) ? a.A0 + rep * NN : dS + NN;
      double* oS = a.dbuf + ((long)rep * 4 + (k & 1) * 2) * NN;
      double* oA = oS + NN;
      const double* Ha = a.Ha + rep * a.hstride;
      const double* Hb = a.Hb + rep * a.hstride;
      double acc[OPT];
#pragma unroll
      for (int u = 0; u < OPT; ++u) acc[u] = 0.0;
      const bool fk = FT && k >= a.kf;   // this term in float32
      float* foS = FT ? a.dbuf32 + ((long)rep * 4 + (k & 1) * 2) * NN : nullptr;
      float* foA = FT ? foS + NN : nullptr;
      if (fk) {
        // the previous term in float32 (the last float64 term also wrote its float32 copy)
        const float* pS = a.dbuf32 + ((long)rep * 4 + ((k - 1) & 1) * 2) * NN;
        const float* pA = pS + NN;
        const float* Hf = a.hbar32 + rep * NN;
        for (int k0 = 0; k0 < N; k0 += KC) {
          for (int e = tid; e < TS * KC; e += NT) {
            const int r = e / KC, kk = e % KC;
            const int kg = k0 + kk;
            const int ri = I * TS + r, rj = J * TS + r;
            fHi[r * (KC + 1) + kk] = (kg < N && ri < N) ? Hf[(long)ri * N + kg] : 0.0f;
            fHj[r * (KC + 1) + kk] = (kg < N && rj < N) ? Hf[(long)rj * N + kg] : 0.0f;
          }
          for (int e = tid; e < KC * TS; e += NT) {
            const int kk = e / TS, b = e % TS;
            const int kg = k0 + kk;
            const int ci = I * TS + b, cj = J * TS + b;
            float ai = 0.f, aj = 0.f, si = 0.f, sj = 0.f;
            if (kg < N) {
              if (ci < N) {
                ai = pA[(long)kg * N + ci];
                si = pS[(long)kg * N + ci];
              }
              if (cj < N) {
                aj = pA[(long)kg * N + cj];
                sj = pS[(long)kg * N + cj];
              }
            }
            fAi[kk * TSP + b] = ai;
            fAj[kk * TSP + b] = aj;
            fSi[kk * TSP + b] = si;
            fSj[kk * TSP + b] = sj;
          }
          __syncthreads();
#pragma unroll
          for (int u = 0; u < OPT; ++u) {
            const int o = tid + NT * u;
            const int q = o / (TS * TS), e = o % (TS * TS);
            const int ra = e / TS, cb = e % TS;
            const float* Hx = (q == 0 || q == 2) ? fHi : fHj;
            const float* Dx = (q == 0) ? fAj : (q == 1) ? fAi : (q == 2) ? fSj : fSi;
            float s0 = 0.f, s1 = 0.f;
#pragma unroll 8
            for (int kk = 0; kk < KC; kk += 2) {
              s0 = fmaf(Hx[ra * (KC + 1) + kk], Dx[kk * TSP + cb], s0);
              s1 = fmaf(Hx[ra * (KC + 1) + kk + 1], Dx[(kk + 1) * TSP + cb], s1);
            }
            acc[u] += (double)(s0 + s1);
          }
          __syncthreads();
        }
      }
      for (int k0 = 0; k0 < (fk ? 0 : N); k0 += KC) {
        for (int e = tid; e < TS * KC; e += NT) {
          const int r = e / KC, kk = e % KC;
          const int kg = k0 + kk;
          const int ri = I * TS + r, rj = J * TS + r;
          double hi = 0.0, hj = 0.0;
          if (kg < N) {
            // (the caller forms Hbar + V beforehand when a field is on: febar is NULL here)
            if (ri < N) hi = 0.5 * (Ha[(long)ri * N + kg] + Hb[(long)ri * N + kg]);
            if (rj < N) hj = 0.5 * (Ha[(long)rj * N + kg] + Hb[(long)rj * N + kg]);
          }
          Hi[r * (KC + 1) + kk] = hi;
          Hj[r * (KC + 1) + kk] = hj;
          if (wd) {
            const double* Dr = a.D + rep * NN;
            Di[r * (KC + 1) + kk] = (kg < N && ri < N) ? Dr[(long)ri * N + kg] : 0.0;
            Dj[r * (KC + 1) + kk] = (kg < N && rj < N) ? Dr[(long)rj * N + kg] : 0.0;
          }
        }
        for (int e = tid; e < KC * TS; e += NT) {
          const int kk = e / TS, b = e % TS;
          const int kg = k0 + kk;
          const int ci = I * TS + b, cj = J * TS + b;
          double ai = 0, aj = 0, si = 0, sj = 0;
          if (kg < N) {
            if (ci < N) {
              ai = dA[(long)kg * N + ci];
              si = dS[(long)kg * N + ci];
            }
            if (cj < N) {
              aj = dA[(long)kg * N + cj];
              sj = dS[(long)kg * N + cj];
            }
          }
          Ai[kk * TSP + b] = ai;
          Aj[kk * TSP + b] = aj;
          Si[kk * TSP + b] = si;
          Sj[kk * TSP + b] = sj;
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < OPT; ++u) {
          const int o = tid + NT * u;
          const int q = o / (TS * TS), e = o % (TS * TS);
          const int ra = e / TS, cb = e % TS;
          const double* Hx = (q == 0 || q == 2) ? Hi : Hj;
          const double* Dx = (q == 0) ? Aj : (q == 1) ? Ai : (q == 2) ? Sj : Si;
          // two float64 FMA chains (even and odd kk): the chain latency, not the rate, would
          // otherwise bound a thread with one output
          double s0 = acc[u], s1 = 0.0;
#pragma unroll 8
          for (int kk = 0; kk < KC; kk += 2) {
            s0 = fma(Hx[ra * (KC + 1) + kk], Dx[kk * TSP + cb], s0);
            s1 = fma(Hx[ra * (KC + 1) + kk + 1], Dx[(kk + 1) * TSP + cb], s1);
          }
          if (wd) {   // + D S (q = 0, 1) or - D A (q = 2, 3)
            const double* Dd = (q == 0 || q == 2) ? Di : Dj;
            const double* Dy = (q == 0) ? Sj : (q == 1) ? Si : (q == 2) ? Aj : Ai;
            double d0 = 0.0, d1 = 0.0;
#pragma unroll 8
            for (int kk = 0; kk < KC; kk += 2) {
              d0 = fma(Dd[ra * (KC + 1) + kk], Dy[kk * TSP + cb], d0);
              d1 = fma(Dd[ra * (KC + 1) + kk + 1], Dy[(kk + 1) * TSP + cb], d1);
            }
            s1 += (q < 2) ? (d0 + d1) : -(d0 + d1);
          }
          acc[u] = s0 + s1;
        }
        __syncthreads();
      }
#pragma unroll
      for (int u = 0; u < OPT; ++u) {
        const int o = tid + NT * u;
        const int q = o / (TS * TS), e = o % (TS * TS);
        Tt[q * TS * TSP + (e / TS) * TSP + (e % TS)] = acc[u];
      }
      __syncthreads();
      double emax = 0.0;
      for (int e = tid; e < TS * TS; e += NT) {
        const int ra = e / TS, cb = e % TS;
        const int i = I * TS + ra, j = J * TS + cb;
        if (i >= N || j >= N) continue;
        const double t1ij = Tt[0 * TS * TSP + ra * TSP + cb];
        const double t1ji = Tt[1 * TS * TSP + cb * TSP + ra];
        const double t2ij = Tt[2 * TS * TSP + ra * TSP + cb];
        const double t2ji = Tt[3 * TS * TSP + cb * TSP + ra];
        const double ns = c * (t1ij + t1ji);
        const double na = -c * (t2ij - t2ji);
        const long o = (long)i * N + j;
        if (FT && k + 1 >= a.kf) {   // the next term reads this one in float32
          foS[o] = (float)ns;
          foA[o] = (float)na;
        }
        if (!fk) {
          oS[o] = ns;
          oA[o] = na;
        }
        a.S1[rep * NN + o] += ns;
        a.A1[rep * NN + o] += na;
        if (I != J) {
          const long ot = (long)j * N + i;
          if (FT && k + 1 >= a.kf) {
            foS[ot] = (float)ns;
            foA[ot] = (float)-na;
          }
          if (!fk) {
            oS[ot] = ns;
            oA[ot] = -na;
          }
          a.S1[rep * NN + ot] += ns;
          a.A1[rep * NN + ot] -= na;
        }
        emax = fmax(emax, ns * ns + na * na);   // |dP_ij|^2
      }
      emax = block_max(emax, sh);
      if (tid == 0) atomic_max_nonneg(&a.slots[(long)rep * (a.max_terms + 1) + k], emax);
      __syncthreads();
    }
    if (!grid_barrier(a.bar, gridDim.x * (unsigned)k, a.status)) return;
    if (tid == 0) {
      int done = 1;
      for (int r = 0; r < a.nrep; ++r) {
        if (conv[r]) continue;
        const unsigned long long bits = *((volatile unsigned long long*)&a.slots[(long)r * (a.max_terms + 1) + k]);
        const double err = __longlong_as_double((long long)bits);   // max |dP_ij|^2
        bool finished = false;
        if (!(err <= 1e300)) {  // NaN or inf
          if (blockIdx.x == 0) atomicCAS(a.status, 0, (int)RMGTD_EDIVERGED);
          if (blockIdx.x == 0 && a.ctl_out) a.ctl_out[a.rep0 + r].status = RMGTD_EDIVERGED;
          finished = true;
        } else if (err <= a.thrs * a.thrs) {
          finished = true;
        } else if (k >= a.max_terms) {
          if (blockIdx.x == 0) atomicCAS(a.status, 0, (int)RMGTD_ENOTCONVERGED);
          if (blockIdx.x == 0 && a.ctl_out) a.ctl_out[a.rep0 + r].status = RMGTD_ENOTCONVERGED;
          finished = true;
        }
        if (finished) {
          conv[r] = 1;
          if (blockIdx.x == 0 && a.ctl_out) {
            RepCtl& cr = a.ctl_out[a.rep0 + r];
            cr.terms_last = k;
            cr.terms_sum += k;
            cr.terms_max = max(cr.terms_max, k);
          }
        } else {
          done = 0;
        }
      }
      all_done = done;
    }
    __syncthreads();
    if (all_done) break;
  }
}

template <int TS, int NT, bool WD, bool FT>
static int launch_eldyn_tsd(rmgtd_ctx* ctx, EldynArgs& a) {
  const int KC = 32;
  const size_t smem = sizeof(double) * (2 * TS * (KC + 1) + 4 * KC * (TS + 1) + 4 * TS * (TS + 1) +
                                        (a.D ? 2 * TS * (KC + 1) : 0));
  static size_t attr_set = 0;
  if (attr_set < smem) {
    RMGTD_CUDA(ctx, cudaFuncSetAttribute(k_eldyn<TS, NT, WD, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    attr_set = smem;
  }
  int per_sm = 0;
  RMGTD_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_eldyn<TS, NT, WD, FT>, NT, smem));
  if (per_sm < 1) return set_error(ctx, RMGTD_ECUDA, "commutator kernel does not fit on an SM");
  const int T = (a.N + TS - 1) / TS;
  const int total = T * (T + 1) / 2 * a.nrep;
  const int grid = std::max(1, std::min(total, per_sm * ctx->num_sms));
  RMGTD_CUDA(ctx, cudaMemsetAsync(a.bar, 0, sizeof(unsigned), ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(a.slots, 0,
                                  sizeof(unsigned long long) * (size_t)a.nrep * (a.max_terms + 1),
                                  ctx->stream));
  void* args[] = {&a};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RMGTD_CUDA(ctx, cudaLaunchKernelExC(&cfg, (const void*)k_eldyn<TS, NT, WD, FT>, args));
  ++ctx->launches;
  return RMGTD_OK;
}

template <int TS, int NT>
static int launch_eldyn_ts(rmgtd_ctx* ctx, EldynArgs& a) {
  if (a.D) return launch_eldyn_tsd<TS, NT, true, false>(ctx, a);
  if (a.kf > 0) return launch_eldyn_tsd<TS, NT, false, true>(ctx, a);
  return launch_eldyn_tsd<TS, NT, false, false>(ctx, a);
}

// Hbar in float32 for the float32 tail: out_r = (Ha_r + Hb_r)/2
__global__ void k_hbar32(long NN, int nrep, const double* __restrict__ Ha, const double* __restrict__ Hb,
                         long hstride, float* __restrict__ out) {
  for (long x = blockIdx.x * (long)blockDim.x + threadIdx.x; x < NN * nrep;
       x += (long)gridDim.x * blockDim.x) {
    const long r = x / NN, o = x - r * NN;
    out[x] = (float)(0.5 * (Ha[r * hstride + o] + Hb[r * hstride + o]));
  }
}

// Commutator series of one replica on one thread-block cluster (N <= 64).  The C CTAs of the
// cluster own consecutive row blocks of the N x N matrices; every CTA keeps a full copy of
// the current term (S_{k-1}, A_{k-1}) in shared memory, forms its rows of T1 = Hbar A_{k-1}
// and T2 = Hbar S_{k-1}, and after a cluster barrier reads the transposed entries T1[j][i],
// T2[j][i] from the owning CTA's shared memory (distributed shared memory), forms its rows of
// S_k, A_k, adds them to P_1 and writes them into every CTA's copy.  Two cluster barriers per
// term and no global-memory round trip: the series of every replica runs on its own cluster
// and the replicas' clusters never wait on one another.
namespace cg = cooperative_groups;

template <int C, bool WD>
__global__ void __launch_bounds__(256, 1) k_eldyn_cluster(EldynArgs a) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int rep = blockIdx.y;
  const int N = a.N;
  const long NN = (long)N * N;
  const int rows = (N + C - 1) / C;
  const int r0 = rank * rows;
  const int nr = max(0, min(rows, N - r0));   // rows owned by this CTA (may be 0)
  const int tid = threadIdx.x, nt = blockDim.x;
  if (a.ctl_in && !a.ctl_in[a.rep0 + rep].active) return;   // whole cluster leaves together

  extern __shared__ double smem[];
  double* Sf = smem;                 // [N][N] current term S_{k-1}
  double* Af = Sf + NN;              // [N][N] current term A_{k-1}
  double* Hr = Af + NN;              // [rows][N] Hbar rows
  double* T1 = Hr + rows * N;        // [rows][N]
  double* T2 = T1 + rows * N;
  double* S1r = T2 + rows * N;       // [rows][N] running P_1
  double* A1r = S1r + rows * N;
  unsigned long long* mx = reinterpret_cast<unsigned long long*>(A1r + rows * N);  // [C]
  double* Dr = reinterpret_cast<double*>(mx + C);   // [rows][N] rows of D (Omega_2 only)
  constexpr bool wd = WD;
  __shared__ unsigned long long shm[8];
  __shared__ double c_sh;

  const double* Ha = a.Ha + rep * a.hstride;
  const double* Hb = a.Hb + rep * a.hstride;
  const double* S0 = a.S0 + rep * NN;
  const double* A0 = a.A0 + rep * NN;
  for (long e = tid; e < NN; e += nt) {
    Sf[e] = S0[e];
    Af[e] = A0[e];
  }
  for (int e = tid; e < nr * N; e += nt) {
    const long o = (long)r0 * N + e;
    Hr[e] = 0.5 * (Ha[o] + Hb[o]) + field_term(a, a.rep0 + rep, o);
    S1r[e] = S0[o];
    A1r[e] = A0[o];
    if (wd) Dr[e] = a.D[rep * NN + o];
  }
  __syncthreads();

  // GB300's float64 rate is ~1/64 of float32: every float64 instruction of the 256 threads
  // costs, so the step tau/k is formed once per term and the maxima of the non-negative
  // |dP_ij|^2 are taken on their bit patterns (integer order = float order; NaN above inf)
  const unsigned long long thr2 = (unsigned long long)__double_as_longlong(a.thrs * a.thrs);
  const unsigned long long big = (unsigned long long)__double_as_longlong(1e300);
  int k = 0;
  int status = 0;
  while (true) {
    ++k;
    if (tid == 0) c_sh = a.tau / (double)k;
    // T1 = Hbar A_{k-1}, T2 = Hbar S_{k-1} on the owned rows.  Two adjacent lanes share an
    // output, each summing half of the m range (two float64 FMA chains of N/2 in flight
    // instead of one of N: the kernel is bound by their latency); the halves are added by a
    // lane exchange.  Uniform trip count, so every lane reaches the exchange.
    {
      const int nout = 2 * nr * N, half = (N + 1) / 2;
      for (int base = 0; base < 2 * nout; base += nt) {
        const int o2 = base + tid;
        const int o = o2 >> 1, hf = o2 & 1;
        double sp = 0.0;
        int q = 0, e = 0;
        if (o < nout) {
          q = o / (nr * N);
          e = o - q * nr * N;
          const int ii = e / N, j = e - ii * N;
          const double* X = q ? Sf : Af;
          const double* h = Hr + ii * N;
          const int m0 = hf ? half : 0, m1 = hf ? N : half;
          for (int m = m0; m < m1; ++m) sp = fma(h[m], X[m * N + j], sp);
          if (wd) {   // + D S (T1) or - D A (T2)
            const double* X2 = q ? Af : Sf;
            const double* dr = Dr + ii * N;
            double sd = 0.0;
            for (int m = m0; m < m1; ++m) sd = fma(dr[m], X2[m * N + j], sd);
            sp += q ? -sd : sd;
          }
        }
        sp += __shfl_xor_sync(0xffffffffu, sp, 1);
        if (o < nout && hf == 0) (q ? T2 : T1)[e] = sp;
      }
    }
    cluster.sync();
    // new terms on the owned rows; broadcast into every CTA's copy
    const double c = c_sh;
    unsigned long long emax = 0;
    for (int e = tid; e < nr * N; e += nt) {
      const int ii = e / N, j = e - ii * N;
      const int i = r0 + ii;
      const int oj = j / rows;
      const int jj = j - oj * rows;
      const double* T1o = cluster.map_shared_rank(T1, oj);
      const double* T2o = cluster.map_shared_rank(T2, oj);
      const double t1ji = T1o[jj * N + i];
      const double t2ji = T2o[jj * N + i];
      const double ns = c * (T1[e] + t1ji);
      const double na = -c * (T2[e] - t2ji);
      S1r[e] += ns;
      A1r[e] += na;
      const double d2 = ns * ns + na * na;   // |dP_ij|^2
      emax = max(emax, (unsigned long long)__double_as_longlong(d2));
      const long off = (long)i * N + j;
      for (int d = 0; d < C; ++d) {
        cluster.map_shared_rank(Sf, d)[off] = ns;
        cluster.map_shared_rank(Af, d)[off] = na;
      }
    }
    for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if ((tid & 31) == 0) shm[tid >> 5] = emax;
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < (nt >> 5); ++w) emax = max(emax, shm[w]);
      for (int d = 0; d < C; ++d) cluster.map_shared_rank(mx, d)[rank] = emax;
    }
    cluster.sync();
    unsigned long long err = 0;
    for (int d = 0; d < C; ++d) err = max(err, mx[d]);
    bool finished = false;
    if (err > big) {                   // inf or NaN (or beyond 1e300)
      status = RMGTD_EDIVERGED;
      finished = true;
    } else if (err <= thr2) {
      finished = true;
    } else if (k >= a.max_terms) {
      status = RMGTD_ENOTCONVERGED;
      finished = true;
    }
    if (finished) break;
  }
  for (int e = tid; e < nr * N; e += nt) {
    const long o = rep * NN + (long)r0 * N + e;
    a.S1[o] = S1r[e];
    a.A1[o] = A1r[e];
  }
  if (a.shat) {   // this CTA's rows of Shat (the rows past N stay zero)
    const int Np = a.Np;
    float* shr = a.shat + (long)(a.rep0 + rep) * Np * Np;
    for (int e = tid; e < nr * Np; e += nt) {
      const int ii = e / Np, j = e - ii * Np, k = r0 + ii;
      double v = 0.0;
      if (j < N && k <= j) {
        const double d = S1r[ii * N + j] - a.Sref[(long)k * N + j];
        v = (k < j) ? 2.0 * d : d;
      }
      shr[(long)k * Np + j] = (float)v;
    }
  }
  if (rank == 0 && tid == 0) {
    if (status) atomicCAS(a.status, 0, status);
    if (a.ctl_out) {
      RepCtl& cr = a.ctl_out[a.rep0 + rep];
      if (status) cr.status = status;
      cr.terms_last = k;
      cr.terms_sum += k;
      cr.terms_max = max(cr.terms_max, k);
    }
  }
}

template <int C>
static int launch_eldyn_cluster(rmgtd_ctx* ctx, EldynArgs& a, size_t smem) {
  const void* fn = a.D ? (const void*)k_eldyn_cluster<C, true> : (const void*)k_eldyn_cluster<C, false>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, a.nrep);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&a};
  RMGTD_CUDA(ctx, cudaLaunchKernelExC(&cfg, fn, args));
  ++ctx->launches;
  return RMGTD_OK;
}

static size_t eldyn_cluster_smem(int N, int C, bool with_d = false) {
  const int rows = (N + C - 1) / C;
  return sizeof(double) * (2 * (size_t)N * N + (with_d ? 6 : 5) * (size_t)rows * N) +
         sizeof(unsigned long long) * C;
}

// Cluster size for the series: 16 CTAs where the device runs such clusters (non-portable
// size), else 8, else 0 (the cooperative kernel runs).
static int eldyn_cluster_size(rmgtd_ctx* ctx) {
  if (ctx->eldyn_cluster >= 0) return ctx->eldyn_cluster;
  ctx->eldyn_cluster = 0;
  for (int C : {16, 8}) {
    // both variants (with and without the Omega_2 rows) get the attributes; the probe uses the
    // larger one
    const size_t smem = eldyn_cluster_smem(ctx->N, C, true);
    const void* fns[2] = {C == 16 ? (const void*)k_eldyn_cluster<16, false>
                                  : (const void*)k_eldyn_cluster<8, false>,
                          C == 16 ? (const void*)k_eldyn_cluster<16, true>
                                  : (const void*)k_eldyn_cluster<8, true>};
    const void* fn = fns[1];
    bool ok = true;
    for (const void* f : fns) {
      if (C == 16 && cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                         cudaSuccess) {
        ok = false;
        break;
      }
      cudaFuncAttributes fa;
      if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) {
        ok = false;
        break;
      }
      if ((size_t)fa.maxDynamicSharedSizeBytes < smem &&
          cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
              cudaSuccess) {
        ok = false;
        break;
      }
    }
    if (!ok) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C, 1);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &cfg) == cudaSuccess && nclusters > 0) {
      ctx->eldyn_cluster = C;
      break;
    }
    cudaGetLastError();
  }
  return ctx->eldyn_cluster;
}

int eldyn(rmgtd_ctx* ctx, const double* Ha, const double* Hb, long hstride, double tau,
          const double* S0, const double* A0, double* S1, double* A1, const RepCtl* ctl_in,
          RepCtl* ctl_out, int rep0, int nreps, float* shat_out, const double* febar,
          const double* D, bool f32_tail) {
  if (nreps > 32) return set_error(ctx, RMGTD_EINVAL, "at most 32 replicas per expansion");
  EldynArgs a;
  a.fM = ctx->M;
  a.febar = febar;
  a.D = D;
  a.kf = 0;
  a.hbar32 = nullptr;
  a.dbuf32 = nullptr;
  a.N = ctx->N;
  a.nrep = nreps;
  a.rep0 = rep0;
  a.Ha = Ha;
  a.Hb = Hb;
  a.hstride = hstride;
  a.tau = tau;
  a.S0 = S0;
  a.A0 = A0;
  a.S1 = S1;
  a.A1 = A1;
  a.dbuf = ctx->dbuf;
  a.ctl_in = ctl_in;
  a.ctl_out = ctl_out;
  a.slots = ctx->errslots;
  a.max_terms = ctx->opt.max_terms;
  a.thrs = ctx->opt.dP_thrs;
  a.bar = ctx->bar;
  a.status = ctx->status;
  // N <= 64: one cluster per replica (no grid barrier); else the cooperative kernel, with
  // small tiles for small N so the float64 work of a term spreads over more SMs
  a.shat = nullptr;
  a.Sref = ctx->Sref;
  a.Np = ((ctx->N + 31) / 32) * 32;
  ctx->shat_fresh = 0;
  if (ctx->N <= 64) {
    const int C = eldyn_cluster_size(ctx);
    if ((C == 16 || C == 8) && shat_out && ctx->Sref) {
      a.shat = shat_out;
      ctx->shat_fresh = 1;   // the density pass that follows skips k_shat32
    }
    if (C == 16) return launch_eldyn_cluster<16>(ctx, a, eldyn_cluster_smem(ctx->N, 16, D));
    if (C == 8) return launch_eldyn_cluster<8>(ctx, a, eldyn_cluster_smem(ctx->N, 8, D));
    ctx->shat_fresh = 0;
  }
  if (a.febar) {   // the cooperative kernel reads plain matrices: Hbar + V into Hx0 first
    if (!ctx->Hx0) return set_error(ctx, RMGTD_EINVAL, "eldyn: field without its scratch");
    int rc = hbar_with_field(ctx, Ha, Hb, hstride, a.febar, rep0, nreps, ctx->Hx0);
    if (rc) return rc;
    a.Ha = a.Hb = ctx->Hx0;
    a.hstride = (long)ctx->N * ctx->N;
    a.febar = nullptr;
  }
  if (f32_tail && !a.D && ctx->hbar32 && ctx->dbuf32) {
    // terms from the third on in float32: a term is ~(tau |Hbar|)^k / k! of P, so its float32
    // rounding stays far below dP_thrs of P; the running P_1 stays float64
    const long NN = (long)ctx->N * ctx->N;
    k_hbar32<<<(int)std::min<long>(ceil_div(NN * nreps, 256), 4L * ctx->num_sms), 256, 0, ctx->stream>>>(
        NN, nreps, a.Ha, a.Hb, a.hstride, ctx->hbar32);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_hbar32");
    a.kf = 3;
    a.hbar32 = ctx->hbar32;
    a.dbuf32 = ctx->dbuf32;
  }
  // GB300's float64 units (~2 FMA per clock and SM) bound the series: pick the tile size
  // whose symmetric tile pairs spread the work of a term most evenly over the SMs (the most
  // loaded SM's share of tile-pair work, items / SMs rounded up times TS^2), small tiles
  // first on ties; 32-point tiles beyond 512 orbitals
  if (ctx->N > 512) return launch_eldyn_ts<32, 256>(ctx, a);
  int best_ts = 16;
  long best = -1;
  for (int ts : {4, 8, 16}) {
    const long T = ceil_div(ctx->N, ts);
    const long items = T * (T + 1) / 2 * nreps;
    const long load = ceil_div(items, (long)ctx->num_sms) * ts * ts;
    if (best < 0 || load < best) {
      best = load;
      best_ts = ts;
    }
  }
  if (best_ts == 4) return launch_eldyn_ts<4, 64>(ctx, a);
  if (best_ts == 8) return launch_eldyn_ts<8, 256>(ctx, a);
  return launch_eldyn_ts<16, 256>(ctx, a);
}

// ---------------------------------------------------------------------------------------
// Step bookkeeping.
// H_1 <- 2 H_0 - H_-1 (Algorithm 1's extrapolation) for every replica; reset the control blocks.
// After a failed step of the same rmgtd_step call (sticky `failed`), every replica is
// left inactive so the remaining steps do nothing.
__global__ void k_step_begin(long n, const double* __restrict__ H0, const double* __restrict__ Hm1,
                             const double* __restrict__ Hm2, double* __restrict__ H1, RepCtl* ctl,
                             int nrep, const int* __restrict__ failed, int* status) {
  const int f = *failed;
  if (!f) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x)
      H1[e] = Hm2 ? 3.0 * (H0[e] - Hm1[e]) + Hm2[e] : 2.0 * H0[e] - Hm1[e];
  }
  if (blockIdx.x == 0 && threadIdx.x < nrep) {
    RepCtl& c = ctl[threadIdx.x];
    c.active = f ? 0 : 1;
    c.passes = 0;
    c.terms_last = c.terms_max = c.terms_sum = 0;
    c.status = 0;
    c.H_err = 0.0;
  }
  if (!f && blockIdx.x == 0 && threadIdx.x == 0) *status = 0;
}

// After one DFT evaluation: H_err = max|H_new - H_1| (already in errbits), decide per
// replica whether the SCF loop continues; inside a graph, set the loop's while flag.
__global__ void k_scf_control(RepCtl* ctl, int nrep, const unsigned long long* errbits,
                              double H_thrs, int max_scf, int* status,
                              cudaGraphConditionalHandle cond, int use_cond,
                              unsigned long long* kexec) {
  const int r = threadIdx.x;
  if (r < nrep) {
    RepCtl& c = ctl[r];
    if (c.active) {
      c.passes += 1;
      const double err = __longlong_as_double((long long)errbits[r]);
      c.H_err = err;
      if (c.status != 0) {
        c.active = 0;
      } else if (!(err <= 1e300)) {
        c.status = RMGTD_EDIVERGED;
        c.active = 0;
        atomicCAS(status, 0, (int)RMGTD_EDIVERGED);
      } else if (err <= H_thrs) {
        c.active = 0;
      } else if (c.passes >= max_scf) {
        c.status = RMGTD_ENOTCONVERGED;
        c.active = 0;
        atomicCAS(status, 0, (int)RMGTD_ENOTCONVERGED);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && use_cond) {
    int a = 0;
    for (int q = 0; q < nrep; ++q) a |= ctl[q].active;
    cudaGraphSetConditional(cond, a ? 1u : 0u);
    atomicAdd(&kexec[0], 1ull);
  }
}

// End of a step: if every replica succeeded, H_-1 <- H_0, H_0 <- H_1, P_0 <- P_1
// (Algorithm 1's shift) and count the step; otherwise raise the sticky failure flag.
// Block 0 appends the control blocks to the per-call statistics.
__global__ void k_step_end(long n, double* __restrict__ Hm2, double* __restrict__ Hm1,
                           double* __restrict__ H0,
                           const double* __restrict__ H1, double* __restrict__ S0,
                           double* __restrict__ A0, const double* __restrict__ S1,
                           const double* __restrict__ A1, const RepCtl* __restrict__ ctl, int nrep,
                           int* failed, int* done_steps, RepCtl* stats, int stats_cap,
                           const int* __restrict__ status, long long* step_dev) {
  if (*failed) return;
  int ok = (*status == 0);
  for (int r = 0; r < nrep; ++r) ok &= (ctl[r].status == 0);
  if (ok) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
         e += (long)gridDim.x * blockDim.x) {
      if (Hm2) Hm2[e] = Hm1[e];
      Hm1[e] = H0[e];
      H0[e] = H1[e];
      S0[e] = S1[e];
      A0[e] = A1[e];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int k = *done_steps;
    if (k < stats_cap)
      for (int r = 0; r < nrep; ++r) stats[(long)k * nrep + r] = ctl[r];
    if (ok) {
      *done_steps = k + 1;
      ++*step_dev;   // completed steps of the context (the field's sample index)
    } else {
      *failed = 1;
    }
  }
}

int step_begin(rmgtd_ctx* ctx) {
  const long n = (long)ctx->nrep * ctx->N * ctx->N;
  const int blocks = (int)std::min<long>(ceil_div(n, 256), 2L * ctx->num_sms);
  k_step_begin<<<std::max(blocks, 1), 256, 0, ctx->stream>>>(n, ctx->H0, ctx->Hm1, ctx->Hm2,
                                                              ctx->H1, ctx->ctl, ctx->nrep,
                                                              ctx->failed, ctx->status);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_step_begin");
  return RMGTD_OK;
}

int scf_control(rmgtd_ctx* ctx, const unsigned long long* errbits,
                cudaGraphConditionalHandle cond, int use_cond) {
  k_scf_control<<<1, 32, 0, ctx->stream>>>(ctx->ctl, ctx->nrep, errbits, ctx->opt.H_thrs,
                                           ctx->opt.max_scf, ctx->status, cond, use_cond,
                                           ctx->kexec);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_scf_control");
  return RMGTD_OK;
}

// ebar[r] = (E_r(t_k) + E_r(t_k + dt)) / 2 for the step that starts after k completed steps
// (samples E_r(j dt), j < nsamp[r]; zero past them), followed by the end values
// ebar[3 nrep + 6 r + q] = E_r(t_k), ebar[3 nrep + 6 r + 3 + q] = E_r(t_k + dt) (Omega_2)
__global__ void k_field_ebar(int nrep, int cap, const double* __restrict__ samples,
                             const int* __restrict__ nsamp, const long long* __restrict__ step_dev,
                             double* __restrict__ ebar) {
  const int t = threadIdx.x;
  if (t >= 3 * nrep) return;
  const int r = t / 3, q = t % 3;
  const long long k = *step_dev;
  const double* E = samples + (long)r * cap * 3;
  const double e0 = k < nsamp[r] ? E[3 * k + q] : 0.0;
  const double e1 = k + 1 < nsamp[r] ? E[3 * (k + 1) + q] : 0.0;
  ebar[t] = 0.5 * (e0 + e1);
  ebar[3 * nrep + 6 * r + q] = e0;
  ebar[3 * nrep + 6 * r + 3 + q] = e1;
}

int field_begin(rmgtd_ctx* ctx) {
  if (!ctx->fld_on) return RMGTD_OK;
  k_field_ebar<<<1, 96, 0, ctx->stream>>>(ctx->nrep, ctx->fld_cap, ctx->fld_samples,
                                           ctx->fld_nsamp, ctx->step_dev, ctx->fld_ebar);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_field_ebar");
  return RMGTD_OK;
}

int step_end(rmgtd_ctx* ctx) {
  const long n = (long)ctx->nrep * ctx->N * ctx->N;
  const int blocks = (int)std::min<long>(ceil_div(n, 256), 2L * ctx->num_sms);
  k_step_end<<<std::max(blocks, 1), 256, 0, ctx->stream>>>(
      n, ctx->Hm2, ctx->Hm1, ctx->H0, ctx->H1, ctx->S0, ctx->A0, ctx->S1, ctx->A1, ctx->ctl, ctx->nrep,
      ctx->failed, ctx->done_steps, ctx->stats_dev, ctx->stats_cap, ctx->status, ctx->step_dev);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_step_end");
  return planes_anchor_update(ctx);
}

// ---------------------------------------------------------------------------------------
// Observables per replica: d_q = Tr(S M_q) (q = x,y,z), Tr(S H_core), Tr(S),
// h^3 sum rho V_H, h^3 sum rho eps_xc.  Two stages with fixed-order sums (deterministic).
constexpr int kObs = 7;

__global__ void k_obs_partial(int N, long Ng, const double* __restrict__ S,
                              const double* __restrict__ M, const double* __restrict__ Hc,
                              const double* __restrict__ rho, const double* __restrict__ vh,
                              const double* __restrict__ exc, const double* __restrict__ rho_core,
                              double* __restrict__ part) {
  const int rep = blockIdx.y;
  const long NN = (long)N * N;
  const double* Sr = S + rep * NN;
  const double* rr = rho + rep * Ng;
  const double* vr = vh + rep * Ng;
  const double* er = exc + rep * Ng;
  double q[kObs] = {0, 0, 0, 0, 0, 0, 0};
  const long stride = (long)gridDim.x * blockDim.x;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < NN; e += stride) {
    const double s = Sr[e];
    q[0] += s * M[e];
    q[1] += s * M[NN + e];
    q[2] += s * M[2 * NN + e];
    q[3] += s * Hc[e];
    const int i = (int)(e / N), j = (int)(e % N);
    if (i == j) q[4] += s;
  }
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += stride) {
    const double r = rr[g];
    q[5] += r * vr[g];
    q[6] += (rho_core ? r + rho_core[g] : r) * er[g];   // E_xc of rho + rho_core
  }
  __shared__ double sh[32];
  for (int t = 0; t < kObs; ++t) {
    const double v = block_sum(q[t], sh);
    if (threadIdx.x == 0) part[((long)rep * kObs + t) * gridDim.x + blockIdx.x] = v;
    __syncthreads();
  }
}

__global__ void k_obs_final(int nblk, const double* __restrict__ part, double h3, double E_ion,
                            double* __restrict__ obs) {
  const int rep = blockIdx.x;
  __shared__ double sh[32];
  double v[kObs];
  for (int t = 0; t < kObs; ++t) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[((long)rep * kObs + t) * nblk + b];
    v[t] = block_sum(s, sh);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* o = obs + 8 * rep;
    o[0] = v[0];
    o[1] = v[1];
    o[2] = v[2];
    o[3] = v[4];                                             // Tr(Re P)
    o[4] = v[3] + 0.5 * h3 * v[5] + h3 * v[6] + E_ion;       // total energy
    o[5] = v[3];                                             // Tr(Re P H_core)
    o[6] = 0.5 * h3 * v[5];                                  // Hartree energy
    o[7] = h3 * v[6];                                        // xc energy
  }
}

int observables(rmgtd_ctx* ctx) {
  const int nblk = ctx->red_blocks;
  k_obs_partial<<<dim3(nblk, ctx->nrep), 256, 0, ctx->stream>>>(
      ctx->N, ctx->Ng, ctx->S0, ctx->M, ctx->Hcore, ctx->rho, ctx->vh, ctx->exc, ctx->rho_core,
      ctx->red_part);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_obs_partial");
  k_obs_final<<<ctx->nrep, 256, 0, ctx->stream>>>(nblk, ctx->red_part, ctx->h3, ctx->E_ion,
                                                  ctx->obs);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_obs_final");
  return RMGTD_OK;
}

// ---------------------------------------------------------------------------------------
// Subspace ground state (set-up): one SCF update of the density matrix inside the orbital
// block.  H (float64, per replica) is diagonalised by parallel cyclic Jacobi rotations
// (round-robin pairing: N/2 disjoint rotations per round, applied to rows, then columns),
// the aufbau density matrix P_new = sum_n f_n w_n w_n^T of the ascending eigenvectors is
// formed, max|P_new - P| is recorded and P <- (1 - alpha) P + alpha P_new.  One block per
// replica; work arrays in global memory (set-up only).
__global__ void __launch_bounds__(1024)
k_subspace_update(int N, const double* __restrict__ H, double* __restrict__ S,
                  const double* __restrict__ f, double alpha, double* __restrict__ work,
                  double* __restrict__ err) {
  const int rep = blockIdx.x;
  const long NN = (long)N * N;
  const double* Hr = H + rep * NN;
  double* Sr = S + rep * NN;
  double* A = work + (long)rep * 3 * NN;
  double* V = A + NN;
  double* Pn = V + NN;
  __shared__ int pp[512], qq[512];
  __shared__ double cc[512], ss[512];
  __shared__ double sh[32];
  __shared__ int ord[1024];
  __shared__ double stop;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long e = tid; e < NN; e += nt) {
    A[e] = Hr[e];
    V[e] = ((e / N) == (e % N)) ? 1.0 : 0.0;
  }
  __syncthreads();
  jacobi_sweeps(N, A, V, pp, qq, cc, ss, sh, &stop);
  if (tid == 0) {  // ascending eigenvalue order (insertion sort, N <= 1024)
    for (int i = 0; i < N; ++i) ord[i] = i;
    for (int i = 1; i < N; ++i) {
      const int o = ord[i];
      const double d = A[(long)o * N + o];
      int j = i - 1;
      while (j >= 0 && A[(long)ord[j] * N + ord[j]] > d) {
        ord[j + 1] = ord[j];
        --j;
      }
      ord[j + 1] = o;
    }
  }
  __syncthreads();
  double emax = 0.0;
  for (long e = tid; e < NN; e += nt) {
    const int i = (int)(e / N), j = (int)(e % N);
    double v = 0.0;
    for (int n = 0; n < N; ++n) {
      const double fn = f[n];
      if (fn != 0.0) v += fn * V[(long)i * N + ord[n]] * V[(long)j * N + ord[n]];
    }
    Pn[e] = v;
    emax = fmax(emax, fabs(v - Sr[e]));
  }
  emax = block_max(emax, sh);
  if (tid == 0) err[rep] = emax;
  __syncthreads();
  for (long e = tid; e < NN; e += nt) Sr[e] = (1.0 - alpha) * Sr[e] + alpha * Pn[e];
}

int subspace_update(rmgtd_ctx* ctx, double alpha, double* err_dev) {
  if (ctx->N > 1024) return set_error(ctx, RMGTD_EINVAL, "subspace ground state needs N <= 1024");
  k_subspace_update<<<ctx->nrep, 1024, 0, ctx->stream>>>(ctx->N, ctx->H1, ctx->S0, ctx->f_dev,
                                                         alpha, ctx->dbuf, err_dev);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_subspace_update");
  return RMGTD_OK;
}

// ---------------------------------------------------------------------------------------
// Orthonormalisation of the starting orbitals: S = h^3 Phi^T Phi = L L^T (Cholesky, one
// block, float64), then Phi <- L^{-1} Phi by forward substitution at every grid point.
__global__ void k_cholesky(int N, double* __restrict__ S, int* status) {
  for (int k = 0; k < N; ++k) {
    __shared__ double d;
    if (threadIdx.x == 0) {
      const double v = S[(long)k * N + k];
      if (!(v > 0.0)) atomicCAS(status, 0, (int)RMGTD_EINVAL);
      d = sqrt(fmax(v, 1e-300));
      S[(long)k * N + k] = d;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < N; i += blockDim.x) S[(long)i * N + k] /= d;
    __syncthreads();
    const long rem = (long)(N - k - 1);
    for (long e = threadIdx.x; e < rem * rem; e += blockDim.x) {
      const int i = k + 1 + (int)(e / rem), j = k + 1 + (int)(e % rem);
      if (j <= i) S[(long)i * N + j] -= S[(long)i * N + k] * S[(long)j * N + k];
    }
    __syncthreads();
  }
}

__global__ void k_forward_subst(int N, long Ng, const double* __restrict__ L,
                                double* __restrict__ phi, double* __restrict__ work) {
  const long g = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (g >= Ng) return;
  double* y = work;  // column-wise scratch [N][Ng] stored at y[i*Ng + g]
  for (int i = 0; i < N; ++i) {
    double s = phi[(long)i * Ng + g];
    for (int j = 0; j < i; ++j) s -= L[(long)i * N + j] * y[(long)j * Ng + g];
    y[(long)i * Ng + g] = s / L[(long)i * N + i];
  }
  for (int i = 0; i < N; ++i) phi[(long)i * Ng + g] = y[(long)i * Ng + g];
}

int forward_subst(rmgtd_ctx* ctx, int N, const double* L, double* X, double* work) {
  k_forward_subst<<<ceil_div(ctx->Ng, 128), 128, 0, ctx->stream>>>(N, ctx->Ng, L, X, work);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_forward_subst");
  return RMGTD_OK;
}

int orthonormalize(rmgtd_ctx* ctx) {
  const int N = ctx->N;
  int rc = gram(ctx, ctx->phi, ctx->phi, nullptr, 0, 1, ctx->h3, nullptr, ctx->Smat, nullptr,
                nullptr, 1, nullptr);
  if (rc) return rc;
  k_cholesky<<<1, 1024, 0, ctx->stream>>>(N, ctx->Smat, ctx->status);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_cholesky");
  double* work = (double*)dev_alloc(ctx, sizeof(double) * (size_t)N * ctx->Ng);
  if (!work) return set_error(ctx, RMGTD_ENOMEM, "orthonormalisation scratch");
  k_forward_subst<<<ceil_div(ctx->Ng, 128), 128, 0, ctx->stream>>>(N, ctx->Ng, ctx->Smat,
                                                                    ctx->phi, work);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_forward_subst");
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  dev_free(ctx, work);
  return RMGTD_OK;
}

}  // namespace rmgtd
