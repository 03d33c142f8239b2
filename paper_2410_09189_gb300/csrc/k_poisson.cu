// Hartree potential: Lap_12 V_H = -4 pi rho on the grid (Section 2.1; Algorithm 1 line 26).
//
// Discrete problem (the same one the kinetic stencil defines): interior unknowns, ghost
// layers holding the monopole + dipole field of rho about the box centre,
//   (-Lap_12^0) V = 4 pi rho + L_ghost(V_b),  V_b(r) = Q/|r| + p.r/|r|^3.
// The ghost term is linear in (Q, p): L_ghost(V_b) = Q G0 + px Gx + py Gy + pz Gz with four
// grid fields G fixed by the grid, formed once at set-up.
//
// Solver: flexible (Polak-Ribiere) conjugate gradients, preconditioned by one symmetric
// multigrid V-cycle in float32 (the paper's multigrid, Section 2.1): cell-centred coarsening
// by 2, 7-point operators at spacing 2^l h, damped Jacobi smoothing (2 pre, 2 post),
// trilinear prolongation and its transpose/8 as restriction; the levels with <= 4096 points
// run inside one block, whose coarsest level is solved exactly.  The float64 path iterates
// on V itself; the mixed path iterates in float32 on the change of V relative to the
// reference potential.  Stopping test, scalars and reductions are float64.
//
// Layout of the launches: stencil kernels run one thread per grid point on a 3-D launch
// grid (32 x 8 threads per x-y tile, blockIdx.z = plane + nz * replica), so no index is
// divided; pointwise vector updates run a fixed number of grid-stride blocks.  Every kernel
// returns at once for replicas whose solve has converged, so a fixed launch sequence (eager
// or inside a CUDA-graph while loop) is correct.
#include <math.h>

#include "rmgtd_internal.cuh"

namespace rmgtd {

constexpr double kPi = 3.14159265358979323846;
constexpr float kJacobiW = 6.0f / 7.0f;
constexpr int kTailMax = 4096;
constexpr int kPre = 2, kPost = 2, kCoarseSweeps = 40;
// relative residual of the float32 correction solve of the mixed path (float32 CG reaches
// ~1e-6-1e-7; the correction is small next to the float64 reference potential)
constexpr double kMixedPoissonTol = 1e-6;
constexpr int kBX = 32, kBY = 8;   // x-y tile of the 3-D launches

struct Grid3 {
  int nx, ny, nz;
  double h;
};

// Reduction partials: slot s of replica r starts at part + (r * 8 + s) * cap.
//   0 (b,b)  1 (r,r)  2 (r,z)  3 (p,Ap)  4..7 moments of rho   5 also (r_new, z_old)
struct Red {
  double* part;
  int cap;
};
__device__ __forceinline__ double* slot(Red R, int rep, int s) {
  return R.part + ((long)rep * 8 + s) * R.cap;
}

__device__ __forceinline__ bool pcg_skip(const PcgState* st, int rep) { return st[rep].done != 0; }

__device__ __forceinline__ double sum_partials(const double* p, int n) {
  // every lane of the calling warp returns the same fixed-order sum
  double s = 0.0;
  for (int b = (threadIdx.x & 31); b < n; b += 32) s += p[b];
  return warp_sum(s);
}

// 3-D launch helpers: thread (ix, iy) of plane iz of replica rep
struct Pt3 {
  int ix, iy, iz, rep;
  bool in;
  int blin;   // linear block id within the replica
  int nblk;   // blocks per replica
};
__device__ __forceinline__ Pt3 pt3(int nx, int ny, int nz) {
  Pt3 p;
  p.ix = blockIdx.x * kBX + threadIdx.x;
  p.iy = blockIdx.y * kBY + threadIdx.y;
  p.iz = blockIdx.z % nz;
  p.rep = blockIdx.z / nz;
  p.in = (p.ix < nx) && (p.iy < ny);
  p.blin = (p.iz * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  p.nblk = gridDim.x * gridDim.y * nz;
  return p;
}
// block sum for 32 x 8 blocks (each y-row is one warp); valid in thread (0, 0)
__device__ __forceinline__ double block_sum_2d(double v, double* sh) {
  v = warp_sum(v);
  __syncthreads();
  if (threadIdx.x == 0) sh[threadIdx.y] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.y == 0) {
    s = (threadIdx.x < kBY) ? sh[threadIdx.x] : 0.0;
    s = warp_sum(s);
  }
  return s;
}

// ---- set-up: ghost response fields G0, Gx, Gy, Gz ------------------------------------------
__global__ void k_ghost_fields(Grid3 G, double* __restrict__ gf) {
  const long Ng = (long)G.nx * G.ny * G.nz;
  const double ih2 = 1.0 / (G.h * G.h);
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng;
       g += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(g % G.nx), iy = (int)((g / G.nx) % G.ny), iz = (int)(g / ((long)G.nx * G.ny));
    const int idx[3] = {ix, iy, iz};
    const int nn[3] = {G.nx, G.ny, G.nz};
    double g0 = 0, gx = 0, gy = 0, gz = 0;
    for (int ax = 0; ax < 3; ++ax) {
      for (int m = 1; m <= kFdRadius; ++m) {
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          const int t = idx[ax] + sgn * m;
          if (t >= 0 && t < nn[ax]) continue;
          int gi[3] = {ix, iy, iz};
          gi[ax] = t;
          const double x = axis_coord(gi[0], G.nx, G.h), y = axis_coord(gi[1], G.ny, G.h),
                       z = axis_coord(gi[2], G.nz, G.h);
          const double r2 = x * x + y * y + z * z;
          const double r = sqrt(r2);
          const double c = fd_coef(m) * ih2;
          g0 += c / r;
          const double c3 = c / (r2 * r);
          gx += c3 * x;
          gy += c3 * y;
          gz += c3 * z;
        }
      }
    }
    gf[g] = g0;
    gf[Ng + g] = gx;
    gf[2 * Ng + g] = gy;
    gf[3 * Ng + g] = gz;
  }
}

// ---- multipole moments of rho (or rho - rho_ref): partials into slots 4..7 ------------------
__global__ void __launch_bounds__(kBX* kBY)
k_moments(Grid3 G, const double* __restrict__ rho, const double* __restrict__ rho_ref, Red R,
          const RepCtl* __restrict__ ctl) {
  const Pt3 p = pt3(G.nx, G.ny, G.nz);
  if (ctl && !ctl[p.rep].active) return;
  double q[4] = {0, 0, 0, 0};
  if (p.in) {
    const long Ng = (long)G.nx * G.ny * G.nz;
    const long g = ((long)p.iz * G.ny + p.iy) * G.nx + p.ix;
    const double v = rho_ref ? rho[p.rep * Ng + g] - rho_ref[g] : rho[p.rep * Ng + g];
    q[0] = v;
    q[1] = v * axis_coord(p.ix, G.nx, G.h);
    q[2] = v * axis_coord(p.iy, G.ny, G.h);
    q[3] = v * axis_coord(p.iz, G.nz, G.h);
  }
  __shared__ double sh[kBY];
  for (int t = 0; t < 4; ++t) {
    const double s = block_sum_2d(q[t], sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) slot(R, p.rep, 4 + t)[p.blin] = s;
  }
}

// ---- the 12th-order operator A = -Lap_12 with zero ghosts -------------------------------
template <typename V>
__device__ __forceinline__ V apply_A12(const V* __restrict__ x, int ix, int iy, int iz, int nx,
                                       int ny, int nz, V ih2) {
  const long plane = (long)nx * ny;
  const long g = (long)iz * plane + (long)iy * nx + ix;
  V s = (V)(3.0 * fd_coef(0)) * x[g];
#pragma unroll
  for (int m = 1; m <= kFdRadius; ++m) {
    V t = 0;
    if (ix + m < nx) t += x[g + m];
    if (ix - m >= 0) t += x[g - m];
    if (iy + m < ny) t += x[g + (long)m * nx];
    if (iy - m >= 0) t += x[g - (long)m * nx];
    if (iz + m < nz) t += x[g + (long)m * plane];
    if (iz - m >= 0) t += x[g - (long)m * plane];
    s = fma((V)fd_coef(m), t, s);
  }
  return -s * ih2;
}

// b = 4 pi (rho - rho_ref) + Q G0 + p.G (moments from k_moments, `nmom` partials); r = b - A x;
// partials of (b,b) (slot 0) and (r,r) (slot 1)
template <typename V>
__global__ void __launch_bounds__(kBX* kBY)
k_pcg_init(Grid3 G, const double* __restrict__ rho, const double* __restrict__ rho_ref,
           const double* __restrict__ gf, const V* __restrict__ x, V* __restrict__ b,
           V* __restrict__ r, Red R, int nmom, int zero_bc, const RepCtl* __restrict__ ctl) {
  const Pt3 p = pt3(G.nx, G.ny, G.nz);
  if (ctl && !ctl[p.rep].active) return;
  __shared__ double mom[4];
  __shared__ double sh[kBY];
  if (threadIdx.y == 0) {
    for (int t = 0; t < 4; ++t) {
      const double s = sum_partials(slot(R, p.rep, 4 + t), nmom);
      if (threadIdx.x == 0) mom[t] = s;
    }
  }
  __syncthreads();
  const double h3 = G.h * G.h * G.h;
  const double Q = zero_bc ? 0.0 : h3 * mom[0], px = zero_bc ? 0.0 : h3 * mom[1],
               py = zero_bc ? 0.0 : h3 * mom[2], pz = zero_bc ? 0.0 : h3 * mom[3];
  const long Ng = (long)G.nx * G.ny * G.nz;
  double bb = 0.0, rr = 0.0;
  if (p.in) {
    const long g = ((long)p.iz * G.ny + p.iy) * G.nx + p.ix;
    const double dr = rho_ref ? rho[p.rep * Ng + g] - rho_ref[g] : rho[p.rep * Ng + g];
    double bd = 4.0 * kPi * dr;
    bd += Q * gf[g] + px * gf[Ng + g] + py * gf[2 * Ng + g] + pz * gf[3 * Ng + g];
    const V bv = (V)bd;
    b[p.rep * Ng + g] = bv;
    const V rv = bv - apply_A12<V>(x + p.rep * Ng, p.ix, p.iy, p.iz, G.nx, G.ny, G.nz,
                                   (V)(1.0 / (G.h * G.h)));
    r[p.rep * Ng + g] = rv;
    bb = (double)bv * (double)bv;
    rr = (double)rv * (double)rv;
  }
  bb = block_sum_2d(bb, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) slot(R, p.rep, 0)[p.blin] = bb;
  rr = block_sum_2d(rr, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) slot(R, p.rep, 1)[p.blin] = rr;
}

// Ap = A p and partials of (p, Ap) into slot 3
template <typename V>
__global__ void __launch_bounds__(kBX* kBY)
k_pcg_Ap(Grid3 G, const V* __restrict__ pv, V* __restrict__ Ap, Red R,
         const PcgState* __restrict__ st) {
  const Pt3 p = pt3(G.nx, G.ny, G.nz);
  if (pcg_skip(st, p.rep)) return;
  __shared__ double sh[kBY];
  double s = 0.0;
  if (p.in) {
    const long Ng = (long)G.nx * G.ny * G.nz;
    const long g = ((long)p.iz * G.ny + p.iy) * G.nx + p.ix;
    const V* pr = pv + p.rep * Ng;
    const V a = apply_A12<V>(pr, p.ix, p.iy, p.iz, G.nx, G.ny, G.nz, (V)(1.0 / (G.h * G.h)));
    Ap[p.rep * Ng + g] = a;
    s = (double)pr[g] * (double)a;
  }
  s = block_sum_2d(s, sh);
  if (threadIdx.x == 0 && threadIdx.y == 0) slot(R, p.rep, 3)[p.blin] = s;
}

__global__ void k_pcg_state_init(PcgState* st, Red R, int nblk, double tol,
                                 const RepCtl* __restrict__ ctl, int nrep) {
  const int rep = threadIdx.x >> 5;  // one warp per replica
  if (rep >= nrep) return;
  const bool act = !ctl || ctl[rep].active;
  const double bb = sum_partials(slot(R, rep, 0), nblk);
  const double rr = sum_partials(slot(R, rep, 1), nblk);
  if ((threadIdx.x & 31) == 0) {
    PcgState& s = st[rep];
    s.bb = bb;
    s.rr = rr;
    s.cur = 0;
    s.it = 0;
    s.status = 0;
    s.done = (!act || rr <= tol * tol * bb) ? 1 : 0;
    s.rz[0] = s.rz[1] = 0.0;
  }
}

// (r, z) partials into slot 2 (grid-stride, gridDim.x partials); p = z when `first`
template <typename V>
__global__ void k_pcg_rz(long Ng, const V* __restrict__ r, const V* __restrict__ z,
                         V* __restrict__ p, int first, Red R, const PcgState* __restrict__ st) {
  const int rep = blockIdx.y;
  if (pcg_skip(st, rep)) return;
  double s = 0.0;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng;
       g += (long)gridDim.x * blockDim.x) {
    const V zv = z[rep * Ng + g];
    s += (double)r[rep * Ng + g] * (double)zv;
    if (first) p[rep * Ng + g] = zv;
  }
  __shared__ double sh[32];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) slot(R, rep, 2)[blockIdx.x] = s;
}

// store the first (r, z); inside a graph, arm the CG while loop that follows (a nested
// loop's flag is not reset between executions of the enclosing body)
__global__ void k_pcg_rz_store(PcgState* st, Red R, int nblk, int nrep,
                               cudaGraphConditionalHandle cond, int use_cond) {
  const int rep = threadIdx.x >> 5;
  if (rep < nrep && !st[rep].done) {
    const double s = sum_partials(slot(R, rep, 2), nblk);
    if ((threadIdx.x & 31) == 0) st[rep].rz[st[rep].cur] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0 && use_cond) {
    int a = 0;
    for (int r = 0; r < nrep; ++r) a |= (st[r].done == 0);
    cudaGraphSetConditional(cond, a ? 1u : 0u);
  }
}

// alpha = rz / (p,Ap) (slot 3, `nap` partials); x += alpha p; r -= alpha Ap; partials of
// (r,r) (slot 1) and (r_new, z_old) (slot 5), gridDim.x each
template <typename V>
__global__ void k_pcg_xr(long Ng, V* __restrict__ x, V* __restrict__ r, const V* __restrict__ p,
                         const V* __restrict__ Ap, const V* __restrict__ z, Red R, int nap,
                         const PcgState* __restrict__ st) {
  const int rep = blockIdx.y;
  if (pcg_skip(st, rep)) return;
  __shared__ double alpha;
  if (threadIdx.x < 32) {
    const double pAp = sum_partials(slot(R, rep, 3), nap);
    if (threadIdx.x == 0) alpha = st[rep].rz[st[rep].cur] / pAp;
  }
  __syncthreads();
  const V a = (V)alpha;
  double s = 0.0, t = 0.0;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng;
       g += (long)gridDim.x * blockDim.x) {
    const long e = rep * Ng + g;
    x[e] = fma(a, p[e], x[e]);
    const V rv = fma(-a, Ap[e], r[e]);
    r[e] = rv;
    s += (double)rv * (double)rv;
    t += (double)rv * (double)z[e];
  }
  __shared__ double sh[32];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) slot(R, rep, 1)[blockIdx.x] = s;
  __syncthreads();
  t = block_sum(t, sh);
  if (threadIdx.x == 0) slot(R, rep, 5)[blockIdx.x] = t;
}

__global__ void k_pcg_check(PcgState* st, Red R, int nblk, double tol, int max_it, int nrep,
                            int* status) {
  const int rep = threadIdx.x >> 5;
  if (rep >= nrep || st[rep].done) return;
  const double rr = sum_partials(slot(R, rep, 1), nblk);
  if ((threadIdx.x & 31) == 0) {
    PcgState& s = st[rep];
    s.rr = rr;
    if (!(rr <= 1e300)) {
      s.done = 1;
      s.status = RMGTD_EDIVERGED;
      atomicCAS(status, 0, (int)RMGTD_EDIVERGED);
    } else if (rr <= tol * tol * s.bb) {
      s.done = 1;
    } else if (s.it + 1 >= max_it) {
      s.done = 1;
      s.status = RMGTD_ENOTCONVERGED;
      atomicCAS(status, 0, (int)RMGTD_ENOTCONVERGED);
    }
  }
}

// beta = ((r,z_new) - (r,z_old)) / rz_old (Polak-Ribiere); p = z + beta p
template <typename V>
__global__ void k_pcg_p(long Ng, const V* __restrict__ z, V* __restrict__ p, Red R, int nblk,
                        const PcgState* __restrict__ st) {
  const int rep = blockIdx.y;
  if (pcg_skip(st, rep)) return;
  __shared__ double beta;
  if (threadIdx.x < 32) {
    const double rzn = sum_partials(slot(R, rep, 2), nblk);
    const double rzo = sum_partials(slot(R, rep, 5), nblk);
    if (threadIdx.x == 0) beta = (rzn - rzo) / st[rep].rz[st[rep].cur];
  }
  __syncthreads();
  const V bt = (V)beta;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng;
       g += (long)gridDim.x * blockDim.x) {
    const long e = rep * Ng + g;
    p[e] = fma(bt, p[e], z[e]);
  }
}

// end of one CG iteration: store (r,z), advance, and (inside a graph) set the while flag
__global__ void k_pcg_end(PcgState* st, Red R, int nblk, int nrep, int* any_active,
                          cudaGraphConditionalHandle cond, int use_cond,
                          unsigned long long* kexec) {
  const int rep = threadIdx.x >> 5;
  if (rep < nrep && !st[rep].done) {
    const double rz = sum_partials(slot(R, rep, 2), nblk);
    if ((threadIdx.x & 31) == 0) {
      PcgState& s = st[rep];
      s.cur ^= 1;
      s.rz[s.cur] = rz;
      s.it += 1;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0;
    for (int r = 0; r < nrep; ++r) a |= (*((volatile int*)&st[r].done) == 0);
    if (any_active) *any_active = a;
    if (use_cond) {
      cudaGraphSetConditional(cond, a ? 1u : 0u);
      atomicAdd(&kexec[1], 1ull);
    }
  }
}

// ---- multigrid V-cycle in float32 (7-point operators, zero Dirichlet ghosts) ---------------
__device__ __forceinline__ float lap7f(const float* __restrict__ x, int ix, int iy, int iz,
                                       int nx, int ny, int nz, float* center) {
  const long plane = (long)nx * ny;
  const long g = (long)iz * plane + (long)iy * nx + ix;
  const float c = x[g];
  float s = 0.0f;
  if (ix + 1 < nx) s += x[g + 1];
  if (ix > 0) s += x[g - 1];
  if (iy + 1 < ny) s += x[g + nx];
  if (iy > 0) s += x[g - nx];
  if (iz + 1 < nz) s += x[g + plane];
  if (iz > 0) s += x[g - plane];
  *center = c;
  return 6.0f * c - s;  // h^2 * (-Lap_7 x)
}

// one damped-Jacobi sweep: xo = xi + w h^2/6 (b - A xi); first: xi = 0; b64 != NULL: b is
// read from the float64 residual and stored as float in bf; out64 != NULL: result to it
__global__ void __launch_bounds__(kBX* kBY)
k_mg_jacobi(Grid3 G, const float* __restrict__ xi, float* __restrict__ xo, float* __restrict__ bf,
            const double* __restrict__ b64, int first, double* __restrict__ out64,
            const PcgState* __restrict__ st) {
  const Pt3 p = pt3(G.nx, G.ny, G.nz);
  if (pcg_skip(st, p.rep) || !p.in) return;
  const long n = (long)G.nx * G.ny * G.nz;
  const float h2 = (float)(G.h * G.h), ih2 = 1.0f / h2;
  const long g = ((long)p.iz * G.ny + p.iy) * G.nx + p.ix;
  const long e = p.rep * n + g;
  float bv;
  if (b64) {
    bv = (float)b64[e];
    bf[e] = bv;
  } else {
    bv = bf[e];
  }
  float v;
  if (first) {
    v = kJacobiW * h2 / 6.0f * bv;
  } else {
    float c;
    const float ax = lap7f(xi + p.rep * n, p.ix, p.iy, p.iz, G.nx, G.ny, G.nz, &c) * ih2;
    v = c + kJacobiW * h2 / 6.0f * (bv - ax);
  }
  if (out64)
    out64[e] = (double)v;
  else
    xo[e] = v;
}

// Two damped-Jacobi sweeps from x = 0 in one pass: x2 = c (2 b - c A b), c = w h^2/6.
// b64: the fine-level float64 residual, also stored as float into bf.
__global__ void __launch_bounds__(kBX* kBY)
k_mg_pre2(Grid3 G, float* __restrict__ xo, float* __restrict__ bf, const double* __restrict__ b64,
          const PcgState* __restrict__ st) {
  const Pt3 p = pt3(G.nx, G.ny, G.nz);
  if (pcg_skip(st, p.rep) || !p.in) return;
  const long n = (long)G.nx * G.ny * G.nz;
  const float h2 = (float)(G.h * G.h), ih2 = 1.0f / h2;
  const float c = kJacobiW * h2 / 6.0f;
  const long plane = (long)G.nx * G.ny;
  const long g = (long)p.iz * plane + (long)p.iy * G.nx + p.ix;
  const long e = p.rep * n + g;
  float bc, s = 0.0f;
  if (b64) {
    const double* b = b64 + p.rep * n;
    bc = (float)b[g];
    if (p.ix + 1 < G.nx) s += (float)b[g + 1];
    if (p.ix > 0) s += (float)b[g - 1];
    if (p.iy + 1 < G.ny) s += (float)b[g + G.nx];
    if (p.iy > 0) s += (float)b[g - G.nx];
    if (p.iz + 1 < G.nz) s += (float)b[g + plane];
    if (p.iz > 0) s += (float)b[g - plane];
    bf[e] = bc;
  } else {
    const float* b = bf + p.rep * n;
    bc = b[g];
    if (p.ix + 1 < G.nx) s += b[g + 1];
    if (p.ix > 0) s += b[g - 1];
    if (p.iy + 1 < G.ny) s += b[g + G.nx];
    if (p.iy > 0) s += b[g - G.nx];
    if (p.iz + 1 < G.nz) s += b[g + plane];
    if (p.iz > 0) s += b[g - plane];
  }
  const float Ab = (6.0f * bc - s) * ih2;
  xo[e] = c * (2.0f * bc - c * Ab);
}

__global__ void __launch_bounds__(kBX* kBY)
k_mg_residual(Grid3 G, const float* __restrict__ x, const float* __restrict__ b,
              float* __restrict__ r, const PcgState* __restrict__ st) {
  const Pt3 p = pt3(G.nx, G.ny, G.nz);
  if (pcg_skip(st, p.rep) || !p.in) return;
  const long n = (long)G.nx * G.ny * G.nz;
  const float ih2 = (float)(1.0 / (G.h * G.h));
  const long g = ((long)p.iz * G.ny + p.iy) * G.nx + p.ix;
  float c;
  r[p.rep * n + g] = b[p.rep * n + g] - lap7f(x + p.rep * n, p.ix, p.iy, p.iz, G.nx, G.ny, G.nz, &c) * ih2;
}

// trilinear (cell-centred) weights along one axis: fine child f = 2I + a takes 3/4 from I
// and 1/4 from I-1 (a = 0) or I+1 (a = 1)
__device__ __forceinline__ void tri_w(int f, int nc, int* c0, int* c1, float* w0, float* w1) {
  const int I = f >> 1;
  *c0 = I;
  *w0 = 0.75f;
  const int nb = (f & 1) ? I + 1 : I - 1;
  if (nb >= 0 && nb < nc) {
    *c1 = nb;
    *w1 = 0.25f;
  } else {
    *c1 = I;
    *w1 = 0.0f;
  }
}

__device__ __forceinline__ float restrict_point(const float* __restrict__ r, int I, int J, int K,
                                                int nx, int ny, int nz) {
  float s = 0.0f;
  for (int dz = -1; dz <= 2; ++dz) {
    const int fz = 2 * K + dz;
    if (fz < 0 || fz >= nz) continue;
    const float wz = (dz == 0 || dz == 1) ? 0.75f : 0.25f;
    for (int dy = -1; dy <= 2; ++dy) {
      const int fy = 2 * J + dy;
      if (fy < 0 || fy >= ny) continue;
      const float wy = (dy == 0 || dy == 1) ? 0.75f : 0.25f;
      for (int dx = -1; dx <= 2; ++dx) {
        const int fx = 2 * I + dx;
        if (fx < 0 || fx >= nx) continue;
        const float wx = (dx == 0 || dx == 1) ? 0.75f : 0.25f;
        s += wx * wy * wz * r[((long)fz * ny + fy) * nx + fx];
      }
    }
  }
  return 0.125f * s;
}

__device__ __forceinline__ float prolong_point(const float* __restrict__ xc, int fx, int fy, int fz,
                                               int cx, int cy, int cz) {
  int x0, x1, y0, y1, z0, z1;
  float wx0, wx1, wy0, wy1, wz0, wz1;
  tri_w(fx, cx, &x0, &x1, &wx0, &wx1);
  tri_w(fy, cy, &y0, &y1, &wy0, &wy1);
  tri_w(fz, cz, &z0, &z1, &wz0, &wz1);
  auto at = [&](int i, int j, int k) { return xc[((long)k * cy + j) * cx + i]; };
  return wz0 * (wy0 * (wx0 * at(x0, y0, z0) + wx1 * at(x1, y0, z0)) +
                wy1 * (wx0 * at(x0, y1, z0) + wx1 * at(x1, y1, z0))) +
         wz1 * (wy0 * (wx0 * at(x0, y0, z1) + wx1 * at(x1, y0, z1)) +
                wy1 * (wx0 * at(x0, y1, z1) + wx1 * at(x1, y1, z1)));
}

// x <- x + P xc, then one damped-Jacobi sweep on the corrected x, in one pass: the
// corrected values of the 6 neighbours are formed on the fly.  Result into xo.
__global__ void __launch_bounds__(kBX* kBY)
k_mg_prolong_sweep(Grid3 F, Grid3 C, const float* __restrict__ xc, const float* __restrict__ x,
                   float* __restrict__ xo, const float* __restrict__ b,
                   const PcgState* __restrict__ st) {
  const Pt3 p = pt3(F.nx, F.ny, F.nz);
  if (pcg_skip(st, p.rep) || !p.in) return;
  const long nf = (long)F.nx * F.ny * F.nz, nc = (long)C.nx * C.ny * C.nz;
  const float* xcr = xc + p.rep * nc;
  const float* xr = x + p.rep * nf;
  const float h2 = (float)(F.h * F.h);
  const long plane = (long)F.nx * F.ny;
  const int fx = p.ix, fy = p.iy, fz = p.iz;
  const long g = (long)fz * plane + (long)fy * F.nx + fx;
  auto corr = [&](int ax, int ay, int az, long gg) {
    return xr[gg] + prolong_point(xcr, ax, ay, az, C.nx, C.ny, C.nz);
  };
  const float c0 = corr(fx, fy, fz, g);
  float s = 0.0f;
  if (fx + 1 < F.nx) s += corr(fx + 1, fy, fz, g + 1);
  if (fx > 0) s += corr(fx - 1, fy, fz, g - 1);
  if (fy + 1 < F.ny) s += corr(fx, fy + 1, fz, g + F.nx);
  if (fy > 0) s += corr(fx, fy - 1, fz, g - F.nx);
  if (fz + 1 < F.nz) s += corr(fx, fy, fz + 1, g + plane);
  if (fz > 0) s += corr(fx, fy, fz - 1, g - plane);
  const float ax = (6.0f * c0 - s) / h2;
  xo[p.rep * nf + g] = c0 + kJacobiW * h2 / 6.0f * (b[p.rep * nf + g] - ax);
}

// coarse b = (1/8) P^T r (launched over the coarse grid)
__global__ void __launch_bounds__(kBX* kBY)
k_mg_restrict(Grid3 F, Grid3 C, const float* __restrict__ rf, float* __restrict__ bc,
              const PcgState* __restrict__ st) {
  const Pt3 p = pt3(C.nx, C.ny, C.nz);
  if (pcg_skip(st, p.rep) || !p.in) return;
  const long nf = (long)F.nx * F.ny * F.nz, nc = (long)C.nx * C.ny * C.nz;
  const long g = ((long)p.iz * C.ny + p.iy) * C.nx + p.ix;
  bc[p.rep * nc + g] = restrict_point(rf + p.rep * nf, p.ix, p.iy, p.iz, F.nx, F.ny, F.nz);
}

// ---- coarse tail of the V-cycle inside one block (levels with <= kTailMax points) ---------
struct TailLevels {
  int nl;
  int nx[12], ny[12], nz[12];
  float h[12];
};

__device__ void tail_jacobi(const TailLevels& L, int l, float* x, float* t, const float* b,
                            int first) {
  const int nx = L.nx[l], ny = L.ny[l], nz = L.nz[l];
  const long n = (long)nx * ny * nz;
  const float h2 = L.h[l] * L.h[l];
  for (long g = threadIdx.x; g < n; g += blockDim.x) {
    if (first) {
      t[g] = kJacobiW * h2 / 6.0f * b[g];
    } else {
      const int ix = (int)(g % nx), iy = (int)((g / nx) % ny), iz = (int)(g / ((long)nx * ny));
      float c;
      const float ax = lap7f(x, ix, iy, iz, nx, ny, nz, &c) / h2;
      t[g] = c + kJacobiW * h2 / 6.0f * (b[g] - ax);
    }
  }
  __syncthreads();
  for (long g = threadIdx.x; g < n; g += blockDim.x) x[g] = t[g];
  __syncthreads();
}

__global__ void k_mg_tail(TailLevels L, const float* __restrict__ b_in, float* __restrict__ x_out,
                          const float* __restrict__ cinv, const PcgState* __restrict__ st) {
  const int rep = blockIdx.x;
  if (pcg_skip(st, rep)) return;
  extern __shared__ float sm[];
  float* xs[12];
  float* bs[12];
  float* ts[12];
  long off = 0;
  for (int l = 0; l < L.nl; ++l) {
    const long n = (long)L.nx[l] * L.ny[l] * L.nz[l];
    xs[l] = sm + off;
    bs[l] = sm + off + n;
    ts[l] = sm + off + 2 * n;
    off += 3 * n;
  }
  const long n0 = (long)L.nx[0] * L.ny[0] * L.nz[0];
  for (long g = threadIdx.x; g < n0; g += blockDim.x) bs[0][g] = b_in[rep * n0 + g];
  __syncthreads();
  for (int l = 0; l < L.nl; ++l) {
    const bool coarsest = (l == L.nl - 1);
    if (coarsest && cinv) {
      // exact solve with the precomputed inverse of the coarsest operator
      const int nc = L.nx[l] * L.ny[l] * L.nz[l];
      for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        float a = 0.0f;
        for (int j = 0; j < nc; ++j) a = fmaf(cinv[(long)i * nc + j], bs[l][j], a);
        xs[l][i] = a;
      }
      __syncthreads();
      break;
    }
    const int sweeps = coarsest ? kCoarseSweeps : kPre;
    for (int s = 0; s < sweeps; ++s) tail_jacobi(L, l, xs[l], ts[l], bs[l], s == 0);
    if (coarsest) break;
    const int nx = L.nx[l], ny = L.ny[l], nz = L.nz[l];
    const long n = (long)nx * ny * nz;
    const float ih2 = 1.0f / (L.h[l] * L.h[l]);
    for (long g = threadIdx.x; g < n; g += blockDim.x) {
      const int ix = (int)(g % nx), iy = (int)((g / nx) % ny), iz = (int)(g / ((long)nx * ny));
      float c;
      ts[l][g] = bs[l][g] - lap7f(xs[l], ix, iy, iz, nx, ny, nz, &c) * ih2;
    }
    __syncthreads();
    const int cx = L.nx[l + 1], cy = L.ny[l + 1], cz = L.nz[l + 1];
    const long nc = (long)cx * cy * cz;
    for (long g = threadIdx.x; g < nc; g += blockDim.x) {
      const int I = (int)(g % cx), J = (int)((g / cx) % cy), K = (int)(g / ((long)cx * cy));
      bs[l + 1][g] = restrict_point(ts[l], I, J, K, nx, ny, nz);
    }
    __syncthreads();
  }
  for (int l = L.nl - 2; l >= 0; --l) {
    const int nx = L.nx[l], ny = L.ny[l], nz = L.nz[l];
    const int cx = L.nx[l + 1], cy = L.ny[l + 1], cz = L.nz[l + 1];
    const long n = (long)nx * ny * nz;
    for (long g = threadIdx.x; g < n; g += blockDim.x) {
      const int fx = (int)(g % nx), fy = (int)((g / nx) % ny), fz = (int)(g / ((long)nx * ny));
      xs[l][g] += prolong_point(xs[l + 1], fx, fy, fz, cx, cy, cz);
    }
    __syncthreads();
    for (int s = 0; s < kPost; ++s) tail_jacobi(L, l, xs[l], ts[l], bs[l], 0);
  }
  for (long g = threadIdx.x; g < n0; g += blockDim.x) x_out[rep * n0 + g] = xs[0][g];
}

// ---- set-up: inverse of the coarsest 7-point operator (one block, Gauss-Jordan, float64) ----
__global__ void k_coarse_inverse(int nx, int ny, int nz, double h, double* __restrict__ M,
                                 double* __restrict__ Minv, float* __restrict__ out) {
  const int n = nx * ny * nz;
  for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    const int ix = i % nx, iy = (i / nx) % ny, iz = i / (nx * ny);
    const int jx = j % nx, jy = (j / nx) % ny, jz = j / (nx * ny);
    const int d = abs(ix - jx) + abs(iy - jy) + abs(iz - jz);
    M[e] = (i == j) ? 6.0 / (h * h) : (d == 1 ? -1.0 / (h * h) : 0.0);
    Minv[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  __shared__ double piv;
  for (int k = 0; k < n; ++k) {  // SPD: no pivoting needed
    if (threadIdx.x == 0) piv = M[(long)k * n + k];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      M[(long)k * n + j] /= piv;
      Minv[(long)k * n + j] /= piv;
    }
    __syncthreads();
    for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) {
      const int i = (int)(e / n), j = (int)(e % n);
      if (i == k) continue;
      const double f = M[(long)i * n + k];
      if (j != k) M[e] -= f * M[(long)k * n + j];
      Minv[e] -= f * Minv[(long)k * n + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      if (i != k) M[(long)i * n + k] = 0.0;
    __syncthreads();
  }
  for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) out[e] = (float)Minv[e];
}

// ---- host orchestration ------------------------------------------------------------------
static Grid3 grid_of(const MgLevel& L) { return Grid3{L.nx, L.ny, L.nz, L.h}; }

static dim3 grid3(int nx, int ny, int nz, int nrep) {
  return dim3(ceil_div(nx, kBX), ceil_div(ny, kBY), nz * nrep);
}
static int nblk3(int nx, int ny, int nz) { return ceil_div(nx, kBX) * ceil_div(ny, kBY) * nz; }
static const dim3 kBlock3(kBX, kBY, 1);

static Red red_of(rmgtd_ctx* ctx) { return Red{ctx->red_part, ctx->red_cap}; }

// z = M r, M = one float32 V-cycle.  Level-0 input / output are float64 (r64, z64) or
// float32 (r32, z32: the V-cycle then iterates directly in z32).
static int vcycle(rmgtd_ctx* ctx, const double* r64, double* z64, const float* r32, float* z32,
                  int nrep) {
  const PcgState* st = ctx->pcg;
  const int nl = (int)ctx->mg.size();
  const int tail = ctx->mg_tail_level;  // first tail level (>= 1) or -1
  const int nmulti = (tail >= 0) ? tail : nl;
  cudaStream_t s = ctx->stream;
  for (int l = 0; l < nmulti; ++l) {
    MgLevel& L = ctx->mg[l];
    const Grid3 G = grid_of(L);
    const dim3 gr = grid3(L.nx, L.ny, L.nz, nrep);
    const bool coarsest = (l == nl - 1);
    float* lx = (l == 0 && z32) ? z32 : L.x;
    float* lb = (l == 0 && r32) ? const_cast<float*>(r32) : L.b;
    const double* in64 = (l == 0 && !r32) ? r64 : nullptr;
    double* out64 = (l == 0 && !z32) ? z64 : nullptr;
    if (!coarsest) {
      k_mg_pre2<<<gr, kBlock3, 0, s>>>(G, lx, lb, in64, st);
      ++ctx->launches;
      k_mg_residual<<<gr, kBlock3, 0, s>>>(G, lx, lb, L.t, st);
      ++ctx->launches;
      MgLevel& C = ctx->mg[l + 1];
      k_mg_restrict<<<grid3(C.nx, C.ny, C.nz, nrep), kBlock3, 0, s>>>(G, grid_of(C), L.t, C.b, st);
      ++ctx->launches;
      RMGTD_LAUNCH(ctx, "k_mg_descend");
      continue;
    }
    // coarsest level handled by multi-block sweeps (no single-block tail)
    float* bufs[2] = {lx, L.t};
    int cur = (kCoarseSweeps % 2 == 1) ? 0 : 1;  // the last sweep writes x
    for (int sw = 0; sw < kCoarseSweeps; ++sw) {
      const bool last_out64 = (out64 && sw == kCoarseSweeps - 1);
      k_mg_jacobi<<<gr, kBlock3, 0, s>>>(G, bufs[cur ^ 1], bufs[cur], lb,
                                         sw == 0 ? in64 : nullptr, sw == 0,
                                         last_out64 ? out64 : nullptr, st);
      ++ctx->launches;
      cur ^= 1;
    }
    RMGTD_LAUNCH(ctx, "k_mg_jacobi");
  }
  if (tail >= 0) {
    TailLevels T;
    T.nl = nl - tail;
    for (int l = tail; l < nl; ++l) {
      T.nx[l - tail] = ctx->mg[l].nx;
      T.ny[l - tail] = ctx->mg[l].ny;
      T.nz[l - tail] = ctx->mg[l].nz;
      T.h[l - tail] = (float)ctx->mg[l].h;
    }
    k_mg_tail<<<nrep, 1024, ctx->mg_tail_smem, s>>>(T, ctx->mg[tail].b, ctx->mg[tail].x,
                                                     ctx->mg_cinv, st);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_mg_tail");
  }
  for (int l = std::min(nmulti, nl - 1) - 1; l >= 0; --l) {
    MgLevel& L = ctx->mg[l];
    MgLevel& C = ctx->mg[l + 1];
    const Grid3 G = grid_of(L);
    const dim3 gr = grid3(L.nx, L.ny, L.nz, nrep);
    float* lx = (l == 0 && z32) ? z32 : L.x;
    float* lb = (l == 0 && r32) ? const_cast<float*>(r32) : L.b;
    double* out64 = (l == 0 && !z32) ? z64 : nullptr;
    // coarse correction and the first post-sweep in one kernel (result in L.t), then the
    // second post-sweep back into x (or the float64 output)
    k_mg_prolong_sweep<<<gr, kBlock3, 0, s>>>(G, grid_of(C), C.x, lx, L.t, lb, st);
    ++ctx->launches;
    k_mg_jacobi<<<gr, kBlock3, 0, s>>>(G, L.t, lx, lb, nullptr, 0, out64, st);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_mg_ascend");
  }
  return RMGTD_OK;
}

int setup_multigrid(rmgtd_ctx* ctx) {
  ctx->mg.clear();
  int nx = ctx->nx, ny = ctx->ny, nz = ctx->nz;
  double h = ctx->h;
  while (true) {
    MgLevel L;
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.n = (long)nx * ny * nz;
    L.h = h;
    L.x = L.b = L.t = nullptr;
    ctx->mg.push_back(L);
    if (ctx->mg.size() >= 12) break;
    if ((nx & 1) || (ny & 1) || (nz & 1) || nx < 4 || ny < 4 || nz < 4) break;
    nx /= 2;
    ny /= 2;
    nz /= 2;
    h *= 2.0;
  }
  const int nl = (int)ctx->mg.size();
  ctx->mg_tail_level = -1;
  for (int l = 1; l < nl; ++l)
    if (ctx->mg[l].n <= kTailMax) {
      ctx->mg_tail_level = l;
      break;
    }
  size_t smem = 0;
  if (ctx->mg_tail_level >= 0)
    for (int l = ctx->mg_tail_level; l < nl; ++l) smem += 3 * sizeof(float) * ctx->mg[l].n;
  ctx->mg_tail_smem = smem;
  if (smem > 48 * 1024) {
    RMGTD_CUDA(ctx, cudaFuncSetAttribute(k_mg_tail, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
  }
  for (int l = 0; l < nl; ++l) {
    MgLevel& L = ctx->mg[l];
    const size_t bytes = sizeof(float) * (size_t)ctx->nrep * L.n;
    L.x = (float*)dev_alloc(ctx, bytes);
    L.b = (float*)dev_alloc(ctx, bytes);
    L.t = (float*)dev_alloc(ctx, bytes);
    if (!L.x || !L.b || !L.t) return set_error(ctx, RMGTD_ENOMEM, "multigrid levels");
  }
  ctx->mg_cinv = nullptr;
  if (ctx->mg_tail_level >= 0) {
    const MgLevel& Lc = ctx->mg[nl - 1];
    if (Lc.n <= 512) {
      const size_t n2 = (size_t)Lc.n * Lc.n;
      double* M = (double*)dev_alloc(ctx, sizeof(double) * n2);
      double* Mi = (double*)dev_alloc(ctx, sizeof(double) * n2);
      ctx->mg_cinv = (float*)dev_alloc(ctx, sizeof(float) * n2);
      if (!M || !Mi || !ctx->mg_cinv) return set_error(ctx, RMGTD_ENOMEM, "coarse inverse");
      k_coarse_inverse<<<1, 1024, 0, ctx->stream>>>(Lc.nx, Lc.ny, Lc.nz, Lc.h, M, Mi, ctx->mg_cinv);
      ++ctx->launches;
      RMGTD_LAUNCH(ctx, "k_coarse_inverse");
      RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      dev_free(ctx, M);
      dev_free(ctx, Mi);
    }
  }
  ctx->ghost = (double*)dev_alloc(ctx, sizeof(double) * 4 * (size_t)ctx->Ng);
  if (!ctx->ghost) return set_error(ctx, RMGTD_ENOMEM, "ghost fields");
  const Grid3 G{ctx->nx, ctx->ny, ctx->nz, ctx->h};
  const int bl = (int)std::max<long>(1, std::min<long>(ceil_div(ctx->Ng, kThreads), 65535L));
  k_ghost_fields<<<bl, kThreads, 0, ctx->stream>>>(G, ctx->ghost);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_ghost_fields");
  return RMGTD_OK;
}

// slot capacity of the reduction partials: the larger of the 3-D fine-grid block count and
// the grid-stride block count
int poisson_red_cap(int nx, int ny, int nz, int red_blocks) {
  return std::max(nblk3(nx, ny, nz), red_blocks);
}

// Buffers of one Hartree solve: float64 (the solve of rho itself) or float32 (the change
// of V_H relative to the reference potential, mixed path).
struct PcgBufs {
  bool f32;
  void *x, *b, *r, *z, *p, *Ap;
  const double* rho_ref;
  double tol;
};

static PcgBufs pcg_bufs(rmgtd_ctx* ctx, double* vh, int f32) {
  PcgBufs B;
  B.f32 = f32 != 0;
  if (B.f32) {
    B.x = ctx->dvh32;
    B.b = ctx->pcg32_b;
    B.r = ctx->pcg32_r;
    B.z = ctx->pcg32_z;
    B.p = ctx->pcg32_p;
    B.Ap = ctx->pcg32_Ap;
    B.rho_ref = ctx->rho_ref;
    B.tol = std::max(ctx->opt.poisson_tol, kMixedPoissonTol);
  } else {
    B.x = vh;
    B.b = ctx->pcg_b;
    B.r = ctx->pcg_r;
    B.z = ctx->pcg_z;
    B.p = ctx->pcg_p;
    B.Ap = ctx->pcg_Ap;
    B.rho_ref = nullptr;
    B.tol = ctx->opt.poisson_tol;
  }
  return B;
}

// Start of a Hartree solve: moments, right-hand side, initial residual, first V-cycle.
int hartree_begin(rmgtd_ctx* ctx, const double* rho, double* vh, const RepCtl* ctl, int zero_bc,
                  int nrep, cudaGraphConditionalHandle cond, int use_cond, int f32) {
  const Grid3 G{ctx->nx, ctx->ny, ctx->nz, ctx->h};
  const long Ng = ctx->Ng;
  const int rb = ctx->red_blocks;
  const dim3 g3 = grid3(ctx->nx, ctx->ny, ctx->nz, nrep);
  const int nb3 = nblk3(ctx->nx, ctx->ny, ctx->nz);
  cudaStream_t s = ctx->stream;
  const Red R = red_of(ctx);
  const PcgBufs B = pcg_bufs(ctx, vh, f32);
  k_moments<<<g3, kBlock3, 0, s>>>(G, rho, B.rho_ref, R, ctl);
  ++ctx->launches;
  if (B.f32) {
    k_pcg_init<float><<<g3, kBlock3, 0, s>>>(G, rho, B.rho_ref, ctx->ghost, (float*)B.x,
                                             (float*)B.b, (float*)B.r, R, nb3, zero_bc, ctl);
  } else {
    k_pcg_init<double><<<g3, kBlock3, 0, s>>>(G, rho, nullptr, ctx->ghost, (double*)B.x,
                                              (double*)B.b, (double*)B.r, R, nb3, zero_bc, ctl);
  }
  ++ctx->launches;
  k_pcg_state_init<<<1, 32 * nrep, 0, s>>>(ctx->pcg, R, nb3, B.tol, ctl, nrep);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_pcg_init");
  int rc = B.f32 ? vcycle(ctx, nullptr, nullptr, (float*)B.r, (float*)B.z, nrep)
                 : vcycle(ctx, (double*)B.r, (double*)B.z, nullptr, nullptr, nrep);
  if (rc) return rc;
  const dim3 gf(rb, nrep);
  if (B.f32)
    k_pcg_rz<float><<<gf, kThreads, 0, s>>>(Ng, (float*)B.r, (float*)B.z, (float*)B.p, 1, R,
                                            ctx->pcg);
  else
    k_pcg_rz<double><<<gf, kThreads, 0, s>>>(Ng, (double*)B.r, (double*)B.z, (double*)B.p, 1, R,
                                             ctx->pcg);
  ++ctx->launches;
  k_pcg_rz_store<<<1, 32 * nrep, 0, s>>>(ctx->pcg, R, rb, nrep, cond, use_cond);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_pcg_rz");
  return RMGTD_OK;
}

// One flexible-CG iteration for every replica still iterating; `cond` is the graph
// while-handle to update (use_cond = 0 outside a graph).
int hartree_iteration(rmgtd_ctx* ctx, double* vh, int nrep, cudaGraphConditionalHandle cond,
                      int use_cond, int f32) {
  const Grid3 G{ctx->nx, ctx->ny, ctx->nz, ctx->h};
  const long Ng = ctx->Ng;
  const int rb = ctx->red_blocks;
  const dim3 g3 = grid3(ctx->nx, ctx->ny, ctx->nz, nrep);
  const int nb3 = nblk3(ctx->nx, ctx->ny, ctx->nz);
  const dim3 gf(rb, nrep);
  cudaStream_t s = ctx->stream;
  const Red R = red_of(ctx);
  const PcgBufs B = pcg_bufs(ctx, vh, f32);
  if (B.f32) {
    k_pcg_Ap<float><<<g3, kBlock3, 0, s>>>(G, (float*)B.p, (float*)B.Ap, R, ctx->pcg);
    ++ctx->launches;
    k_pcg_xr<float><<<gf, kThreads, 0, s>>>(Ng, (float*)B.x, (float*)B.r, (float*)B.p,
                                            (float*)B.Ap, (float*)B.z, R, nb3, ctx->pcg);
    ++ctx->launches;
  } else {
    k_pcg_Ap<double><<<g3, kBlock3, 0, s>>>(G, (double*)B.p, (double*)B.Ap, R, ctx->pcg);
    ++ctx->launches;
    k_pcg_xr<double><<<gf, kThreads, 0, s>>>(Ng, (double*)B.x, (double*)B.r, (double*)B.p,
                                             (double*)B.Ap, (double*)B.z, R, nb3, ctx->pcg);
    ++ctx->launches;
  }
  k_pcg_check<<<1, 32 * nrep, 0, s>>>(ctx->pcg, R, rb, B.tol, ctx->opt.poisson_max_iter, nrep,
                                      ctx->status);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_pcg_iteration");
  int rc = B.f32 ? vcycle(ctx, nullptr, nullptr, (float*)B.r, (float*)B.z, nrep)
                 : vcycle(ctx, (double*)B.r, (double*)B.z, nullptr, nullptr, nrep);
  if (rc) return rc;
  if (B.f32) {
    k_pcg_rz<float><<<gf, kThreads, 0, s>>>(Ng, (float*)B.r, (float*)B.z, (float*)B.p, 0, R,
                                            ctx->pcg);
    ++ctx->launches;
    k_pcg_p<float><<<gf, kThreads, 0, s>>>(Ng, (float*)B.z, (float*)B.p, R, rb, ctx->pcg);
    ++ctx->launches;
  } else {
    k_pcg_rz<double><<<gf, kThreads, 0, s>>>(Ng, (double*)B.r, (double*)B.z, (double*)B.p, 0, R,
                                             ctx->pcg);
    ++ctx->launches;
    k_pcg_p<double><<<gf, kThreads, 0, s>>>(Ng, (double*)B.z, (double*)B.p, R, rb, ctx->pcg);
    ++ctx->launches;
  }
  k_pcg_end<<<1, 32 * nrep, 0, s>>>(ctx->pcg, R, rb, nrep, ctx->pcg_any, cond, use_cond,
                                     ctx->kexec);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_pcg_end");
  return RMGTD_OK;
}

// Initial guess of the first Hartree solve of a step: linear extrapolation in time,
// x <- 2 x(t) - x(t - dt), prev <- x(t).  Only the CG starting point changes.
template <typename T>
__global__ void k_extrap(long n, T* __restrict__ x, T* __restrict__ prev,
                         const int* __restrict__ failed) {
  if (*failed) return;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const T t = x[e];
    x[e] = (T)2 * t - prev[e];
    prev[e] = t;
  }
}

int hartree_extrapolate(rmgtd_ctx* ctx) {
  if (!ctx->hartree_xc) return RMGTD_OK;
  const long n = (long)ctx->nrep * ctx->Ng;
  const int bl = (int)std::max<long>(1, std::min<long>(ceil_div(n, kThreads), 65535L));
  if (ctx->mixed)
    k_extrap<float><<<bl, kThreads, 0, ctx->stream>>>(n, ctx->dvh32, ctx->dvh_prev32, ctx->failed);
  else
    k_extrap<double><<<bl, kThreads, 0, ctx->stream>>>(n, ctx->vh, ctx->vh_prev, ctx->failed);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_extrap");
  return RMGTD_OK;
}

// prev <- current (no history yet: the first extrapolation reproduces the current guess)
int hartree_reset_history(rmgtd_ctx* ctx) {
  const long n = (long)ctx->nrep * ctx->Ng;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->vh_prev, ctx->vh, sizeof(double) * n,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
  if (ctx->mixed)
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->dvh_prev32, ctx->dvh32, sizeof(float) * n,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
  return RMGTD_OK;
}

// Eager Hartree solve (host-driven loop, peeking at the convergence flag).
int hartree_dev(rmgtd_ctx* ctx, const double* rho, double* vh, const RepCtl* ctl, int zero_bc,
                int nrep, int f32) {
  int rc = hartree_begin(ctx, rho, vh, ctl, zero_bc, nrep, 0, 0, f32);
  if (rc) return rc;
  for (int it = 0; it < ctx->opt.poisson_max_iter; ++it) {
    rc = hartree_iteration(ctx, vh, nrep, 0, 0, f32);
    if (rc) return rc;
    if ((it & 3) == 3) {
      RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->pcg_any_host, ctx->pcg_any, sizeof(int),
                                      cudaMemcpyDeviceToHost, ctx->stream));
      RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (!*ctx->pcg_any_host) break;
    }
  }
  return RMGTD_OK;
}

}  // namespace rmgtd
