// Propagation of the occupied orbitals on the grid: the complete-grid-basis limit of
// Algorithm 1 (Section 2.2: the propagation holds in any basis; the grid is the complete
// one).  P = sum_n f_n |psi_n><psi_n| is propagated by applying the series of Eq. 33 to the
// orbitals, psi^(k) = (-i dt / k) Hbar psi^(k-1), with Hbar = T + V_ion + V_NL +
// (V_0 + V_1)/2 + sum_q Ebar_q q, inside the same SCF loop on V = V_H + V_xc (in the grid
// basis H_new - H_1 is diagonal, so H_err = max|V_new - V_1|), then a Cholesky
// re-orthonormalisation in float64.  The kick is the pointwise phase e^{-i kappa q}.
//
// Layout: per replica the orbitals are planar complex, [2][nocc][Ng] (real plane, then
// imaginary plane).  The state psi, the series' sum psi_1, the potentials and the
// re-orthonormalisation are float64; the series terms are float64 (FP64 path) or float32
// (mixed path: the terms of a smooth orbital shrink fast, and a term's float32 rounding is
// carried forward by the remaining, unitary, series, so the sum keeps ~1e-7 of |psi|).  One
// fused kernel per term: the 12th-order stencil of both planes, the potential, the KB part
// from per-point projector lists, the running sum and the stopping maximum.  With float64
// terms the sum is psi_1 itself (psi_1 += t); with float32 terms it is a compensated float32
// pair (hi + lo, the two-sum of Knuth), each pass's density is a float32 change on the float64
// density of the step's psi, and psi_1 = psi + hi + lo is formed once, when the SCF loop
// ends: no float64 arithmetic is left per term or per pass (GB300's float64 pipe runs at 1/64
// of its float32 rate).  The host drives the pass loop and queues the terms in batches behind
// a device-side stopping test.
#include <cstring>
#include <utility>

#include "rmgtd_internal.cuh"
#include "tc_common.cuh"

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

// out = 2 a - b (V_1 <- 2 V_0 - V_-1, Algorithm 1's extrapolation on the potential), or with
// c (seed_order 2) the quadratic out = 3 a - 3 b + c (V_1 <- 3 V_0 - 3 V_-1 + V_-2)
__global__ void k_gp_extrap(const double* __restrict__ a, const double* __restrict__ b,
                            const double* __restrict__ c, double* __restrict__ out, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    out[e] = c ? 3.0 * (a[e] - b[e]) + c[e] : 2.0 * a[e] - b[e];
}

// vtot_r = V_ion + (V0_r + V1_r)/2 + sum_q ebar_rq q, in the terms' precision
template <typename T>
__global__ void k_gp_vtot(const double* __restrict__ vion, const double* __restrict__ v0,
                          const double* __restrict__ v1, const double* __restrict__ ebar,
                          T* __restrict__ vtot, long Ng, int nx, int ny, int nz, double h) {
  const int r = blockIdx.y;
  const double ex = ebar[3 * r], ey = ebar[3 * r + 1], ez = ebar[3 * r + 2];
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x) {
    const long o = r * Ng + g;
    double v = vion[g] + 0.5 * (v0[o] + v1[o]);
    if (ex != 0.0 || ey != 0.0 || ez != 0.0)
      v += ex * coord_of(g, 0, nx, ny, nz, h) + ey * coord_of(g, 1, nx, ny, nz, h) +
           ez * coord_of(g, 2, nx, ny, nz, h);
    vtot[o] = (T)v;
  }
}

// the stencil and series coefficients of one term in the terms' precision, formed on the
// host and read by the kernels from their parameter space: cm[m] = a_m (-1/(2h^2)) for the
// 12th-order Laplacian, c0 = 3 a_0 (-1/(2h^2)), c = dt / k.  (Formed in the kernels, the
// float64 products would be recomputed for every plane where registers are short.)
template <typename T>
struct GpTermCoef {
  T cm[kFdRadius + 1];
  T c0;
  T c;
};

template <typename T>
GpTermCoef<T> gp_term_coef(double h, double c) {
  GpTermCoef<T> k{};
  const double cscale = -0.5 / (h * h);
  for (int m = 1; m <= kFdRadius; ++m) k.cm[m] = (T)(fd_coef(m) * cscale);
  k.c0 = (T)(3.0 * fd_coef(0) * cscale);
  k.c = (T)c;
  return k;
}

// start of a pass for the active replicas: t = psi (in the terms' precision) and, with
// float64 terms, psi_1 = psi (psi1 null: float32 terms, whose sum starts at the first term)
template <typename T>
__global__ void k_gp_start(const double* __restrict__ psi, double* __restrict__ psi1,
                           T* __restrict__ t, long rplane, const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (!active[r]) return;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < rplane;
       e += (long)gridDim.x * blockDim.x) {
    const long o = r * rplane + e;
    if (psi1) psi1[o] = psi[o];
    t[o] = (T)psi[o];
  }
}

// s + e = a + b exactly, s = fl(a + b) (Knuth's two-sum: six additions, no branch)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// the series' running sum at element o: float64 terms add to psi_1; float32 terms to the
// pair (hi at o, lo at o + lo_off) by a two-sum, the first term setting it
__device__ __forceinline__ void series_add(double* a, long o, long, double v, bool) { a[o] += v; }
__device__ __forceinline__ void series_add(float* a, long o, long lo_off, float v, bool first) {
  if (first) {
    a[o] = v;
    a[o + lo_off] = 0.f;
    return;
  }
  float s, e;
  two_sum(a[o], v, s, e);
  a[o] = s;
  a[o + lo_off] += e;
}

// after term k: the stopping test of every running series on the device, so that the host
// can queue several terms between read-backs.  ctl = [running][status][terms] per replica;
// a series stops when max|t|^2 <= thr2 (converged), is not finite (diverged) or k reaches
// the term limit; errbits is cleared for the next term.
__global__ void k_gp_series_ctl(int nrep, int k, double thr2, int max_terms, int* __restrict__ ctl,
                                unsigned long long* __restrict__ errbits) {
  for (int r = threadIdx.x; r < nrep; r += blockDim.x) {
    if (!ctl[r]) continue;
    const double m = __longlong_as_double((long long)errbits[r]);
    errbits[r] = 0ull;
    int st = 0;
    bool stop = true;
    if (!(m <= 1e300)) st = RMGTD_EDIVERGED;
    else if (m <= thr2) st = 0;
    else if (k >= max_terms) st = RMGTD_ENOTCONVERGED;
    else stop = false;
    if (stop) {
      ctl[r] = 0;
      ctl[nrep + r] = st;
      ctl[2 * nrep + r] = k;
    }
  }
}

// end of a step with float32 terms (every replica, active null): psi_1 = psi + (hi + lo)
__global__ void k_gp_fold(const double* __restrict__ psi, const float* __restrict__ acc,
                          long lo_off, double* __restrict__ psi1, long rplane,
                          const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < rplane;
       e += (long)gridDim.x * blockDim.x) {
    const long o = r * rplane + e;
    psi1[o] = psi[o] + ((double)acc[o] + (double)acc[o + lo_off]);
  }
}

// KB projections of the real columns j of x (the term planes): coef[j][p] =
// h^3 sum_e beta_p(e) x_j(g_e) over projector p's box, g_e the box entry's grid index.
// Block (p, group of kKbCols columns): each thread takes every blockDim-th entry, four at a
// time (their indexes, values and the kKbCols column values all in flight together), and
// keeps one sum per column: float64 columns in float64, float32 columns in compensated
// float32 (Kahan), summed across the warp as float32 pairs; the warps' sums are then added in
// float64 in a fixed order.  Columns
// of replicas whose series has stopped are skipped (cols_per_rep columns per replica).
constexpr int kKbCols = 4, kKbThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kKbThreads)
k_gp_kb_project(const T* __restrict__ x, long Ng, int ncols, int cols_per_rep,
                const int* __restrict__ sact, const long long* __restrict__ off,
                const int* __restrict__ pt, const T* __restrict__ pv, double h3,
                T* __restrict__ coef) {
  const int p = blockIdx.x, np = gridDim.x, j0 = blockIdx.y * kKbCols;
  const long long e0 = off[p];
  const int nb = (int)(off[p + 1] - e0);
  const int* ptp = pt + e0;
  const T* pvp = pv + e0;
  __shared__ double sh[kKbCols][kKbThreads / 32];
  bool act[kKbCols], any = false;
  const T* xc[kKbCols];
#pragma unroll
  for (int c = 0; c < kKbCols; ++c) {
    const int j = min(j0 + c, ncols - 1);
    act[c] = j0 + c < ncols && sact[j / cols_per_rep];
    any = any || act[c];
    xc[c] = x + (long)j * Ng;
  }
  if (!any) return;   // uniform over the block
  T s[kKbCols], comp[kKbCols];
#pragma unroll
  for (int c = 0; c < kKbCols; ++c) s[c] = comp[c] = (T)0;
  const int step = blockDim.x;
  for (int e = threadIdx.x; e < nb; e += 4 * step) {
    int g[4];
    T b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int eu = e + u * step;
      g[u] = eu < nb ? ptp[eu] : 0;
      b[u] = eu < nb ? pvp[eu] : (T)0;
    }
    T xv[kKbCols][4];
#pragma unroll
    for (int c = 0; c < kKbCols; ++c)
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[c][u] = act[c] ? xc[c][g[u]] : (T)0;
#pragma unroll
    for (int c = 0; c < kKbCols; ++c)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T v = b[u] * xv[c][u];
        if constexpr (sizeof(T) == sizeof(double)) {
          s[c] += v;
        } else {
          const T y = v - comp[c], t = s[c] + y;
          comp[c] = (t - s[c]) - y;
          s[c] = t;
        }
      }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int c = 0; c < kKbCols; ++c) {
    if constexpr (sizeof(T) == sizeof(double)) {
      const double v = warp_sum(s[c]);
      if (lane == 0) sh[c][w] = v;
    } else {   // the warp's sum as a float32 pair (two-sum butterfly), float64 from lane 0
      float hi = s[c], lo = -comp[c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, hi, off);
        const float ol = __shfl_xor_sync(0xffffffffu, lo, off);
        float t, e;
        two_sum(hi, oh, t, e);
        hi = t;
        lo = __fadd_rn(__fadd_rn(lo, ol), e);
      }
      if (lane == 0) sh[c][w] = (double)hi + (double)lo;
    }
  }
  __syncthreads();
  if (w < kKbCols) {
    const int c = w;
    double v = lane < nw ? sh[c][lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0 && j0 + c < ncols) coef[(long)(j0 + c) * np + p] = (T)(h3 * v);
  }
}

// One term of the orbital series for orbital n of replica r over a z-range:
//   t_out = (-i c) (T + V + V_NL) t_in,  sum += t_out,  errbits_r <- max |t_out|^2,
// c = dt / k (the sum: psi_1 for float64 terms, the float32 pair for float32 terms).  Block BX x BY over an x-y tile, marching along z with each thread's z-column
// (both planes) in registers; the x-y neighbourhood of every plane staged in shared memory
// with a 6-point halo (zero outside the grid: Dirichlet ghosts).  The KB part reads the
// point's projector list (E_p beta_p(r)) and the projections of t_in.
template <typename T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
k_gp_term_fused(const T* __restrict__ tin, T* __restrict__ tout, T* __restrict__ acc, long lo_off,
                int first, const T* __restrict__ vtot, const int* __restrict__ kb_row,
                const int* __restrict__ kb_p, const T* __restrict__ kb_w,
                const T* __restrict__ coef, int np, int nocc, int nx, int ny, int nz,
                int zchunk, int nzc, const GpTermCoef<T> kc, const int* __restrict__ sact,
                unsigned long long* __restrict__ errbits) {
  constexpr int R = kFdRadius;
  constexpr int TX = BX + 2 * R, TY = BY + 2 * R;
  __shared__ T sre[TY][TX];
  __shared__ T sim[TY][TX];
  __shared__ double sh[32];
  const int col = blockIdx.z / nzc;   // rep * nocc + n
  const int rep = col / nocc, n = col - rep * nocc;
  if (!sact[rep]) return;             // uniform over the block
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int z0 = (blockIdx.z % nzc) * zchunk, z1 = min(nz, z0 + zchunk);
  const int ix = blockIdx.x * BX + tx, iy = blockIdx.y * BY + ty;
  const bool in_xy = ix < nx && iy < ny;
  const long plane = (long)nx * ny, Ng = plane * nz, oplane = (long)nocc * Ng;
  const long base = (long)rep * 2 * oplane + (long)n * Ng;
  const T* xr = tin + base;
  const T* xi = xr + oplane;
  T* yr = tout + base;
  T* yi = yr + oplane;
  const T* v = vtot + (long)rep * Ng;
  const T* cre = coef + (long)(rep * 2 * nocc + n) * np;          // column re
  const T* cim = coef + (long)(rep * 2 * nocc + nocc + n) * np;   // column im
  T qr[2 * R + 1], qi[2 * R + 1];
#pragma unroll
  for (int k = 0; k < 2 * R; ++k) {
    const int z = z0 - R + k;
    const bool ok = in_xy && z >= 0 && z < nz;
    const long g = (long)z * plane + (long)iy * nx + ix;
    qr[k] = ok ? xr[g] : (T)0;
    qi[k] = ok ? xi[g] : (T)0;
  }
  T emax = (T)0;
  for (int z = z0; z < z1; ++z) {
    {
      const int zz = z + R;
      const bool ok = in_xy && zz < nz;
      const long g = (long)zz * plane + (long)iy * nx + ix;
      qr[2 * R] = ok ? xr[g] : (T)0;
      qi[2 * R] = ok ? xi[g] : (T)0;
    }
    for (int e = tid; e < TX * TY; e += BX * BY) {
      const int ly = e / TX, lx = e - ly * TX;
      const int gx = blockIdx.x * BX + lx - R, gy = blockIdx.y * BY + ly - R;
      const bool corner = (lx < R || lx >= BX + R) && (ly < R || ly >= BY + R);
      T a = (T)0, b = (T)0;
      if (!corner && gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
        const long g = (long)z * plane + (long)gy * nx + gx;
        a = xr[g];
        b = xi[g];
      }
      sre[ly][lx] = a;
      sim[ly][lx] = b;
    }
    __syncthreads();
    if (in_xy) {
      const long g = (long)z * plane + (long)iy * nx + ix;
      T ar = kc.c0 * qr[R], ai = kc.c0 * qi[R];
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const T sr = (sre[ty + R][tx + R + m] + sre[ty + R][tx + R - m]) +
                     (sre[ty + R + m][tx + R] + sre[ty + R - m][tx + R]) + (qr[R + m] + qr[R - m]);
        const T si = (sim[ty + R][tx + R + m] + sim[ty + R][tx + R - m]) +
                     (sim[ty + R + m][tx + R] + sim[ty + R - m][tx + R]) + (qi[R + m] + qi[R - m]);
        ar = fma(kc.cm[m], sr, ar);
        ai = fma(kc.cm[m], si, ai);
      }
      const T vv = v[g];
      ar = fma(vv, qr[R], ar);
      ai = fma(vv, qi[R], ai);
      if (kb_row) {
        T kr = (T)0, ki = (T)0;
        for (int e = kb_row[g]; e < kb_row[g + 1]; ++e) {
          const int p = kb_p[e];
          const T w = kb_w[e];
          kr = fma(w, cre[p], kr);
          ki = fma(w, cim[p], ki);
        }
        ar += kr;
        ai += ki;
      }
      const T nr = kc.c * ai, ni = -kc.c * ar;   // -i c (ar + i ai)
      yr[g] = nr;
      yi[g] = ni;
      series_add(acc, base + g, lo_off, nr, first);
      series_add(acc, base + oplane + g, lo_off, ni, first);
      emax = fmax(emax, nr * nr + ni * ni);   // in the terms' precision (a stopping test)
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) {
      qr[k] = qr[k + 1];
      qi[k] = qi[k + 1];
    }
  }
  const double bm = block_max((double)emax, sh);
  if (tid == 0) atomic_max_nonneg(&errbits[rep], bm);
}

// The same term (float64 terms; float32 terms use k_gp_term_tma2 below) with the x-y tiles
// streamed by TMA: thread 0 keeps kGtS planes of the chunk
// in flight, each a pair of tiles (real, imaginary) of (BX + 16) x (BY + 12) points starting at
// (x0 - 8, y0 - 6) -- the x start rounded down to a 16-byte boundary -- with zero fill outside
// the grid (the Dirichlet ghosts).  Each thread's z-column stays in registers, refilled by a
// coalesced load issued one plane ahead.  One block barrier per plane; waits are bounded
// (status <- ETIMEOUT, the copies in flight are waited for before the block leaves).
constexpr int kGtS = 6;     // planes in flight
constexpr int kGtXO = 8;    // x offset of the interior in a tile

template <typename T, int BX, int BY>
__host__ __device__ constexpr int gt_tile_elems() {
  return (BY + 2 * kFdRadius) * (BX + 2 * kGtXO);
}

template <typename T, int BX, int BY>
__host__ __device__ constexpr size_t gt_smem_bytes() {
  return sizeof(T) * 2 * gt_tile_elems<T, BX, BY>() * kGtS + sizeof(uint64_t) * kGtS + 1024;
}

template <typename T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
k_gp_term_tma(const __grid_constant__ CUtensorMap tm_in, const T* __restrict__ tin,
              T* __restrict__ tout, double* __restrict__ psi1, const T* __restrict__ vtot,
              const int* __restrict__ kb_row, const int* __restrict__ kb_p,
              const T* __restrict__ kb_w, const T* __restrict__ coef, int np, int nocc,
              int nx, int ny, int nz, int zchunk, int nzc, const GpTermCoef<T> kc,
              const int* __restrict__ sact, unsigned long long* __restrict__ errbits,
              int* __restrict__ status) {
  static_assert(sizeof(T) == sizeof(double), "float32 terms use k_gp_term_tma2");
  constexpr int R = kFdRadius;
  constexpr int TW = BX + 2 * kGtXO;            // tile row length
  constexpr int TE = gt_tile_elems<T, BX, BY>();
  constexpr uint32_t kBytes = 2u * TE * sizeof(T);
  extern __shared__ unsigned char gt_raw[];
  unsigned char* gt_smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(gt_raw) + 1023) & ~(uintptr_t)1023);
  T* tiles = reinterpret_cast<T*>(gt_smem);     // [kGtS][2][BY + 2R][TW]
  uint64_t* full = reinterpret_cast<uint64_t*>(gt_smem + sizeof(T) * 2 * TE * kGtS);
  __shared__ double sh[32];
  const int col = blockIdx.z / nzc;   // rep * nocc + n
  const int rep = col / nocc, n = col - rep * nocc;
  if (!sact[rep]) return;             // uniform over the block, before any barrier
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * BX + tx;
  const int z0 = (blockIdx.z % nzc) * zchunk, z1 = min(nz, z0 + zchunk), nzb = z1 - z0;
  const int ix = blockIdx.x * BX + tx, iy = blockIdx.y * BY + ty;
  const bool in_xy = ix < nx && iy < ny;
  const long plane = (long)nx * ny, Ng = plane * nz, oplane = (long)nocc * Ng;
  const long base = (long)rep * 2 * oplane + (long)n * Ng;
  const int cre_col = rep * 2 * nocc + n, cim_col = cre_col + nocc;   // tensor-map columns
  const int xs = blockIdx.x * BX - kGtXO, ys = blockIdx.y * BY - R;
  if (tid == 0) {
    for (int s = 0; s < kGtS; ++s) tc::mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int i = 0; i < min(kGtS, nzb); ++i) {
      T* dst = tiles + (size_t)i * 2 * TE;
      const uint32_t bar = tc::saddr(&full[i]);
      tc::mbar_expect_tx(bar, kBytes);
      tc::tma_load_4d(tc::saddr(dst), &tm_in, xs, ys, z0 + i, cre_col, bar);
      tc::tma_load_4d(tc::saddr(dst + TE), &tm_in, xs, ys, z0 + i, cim_col, bar);
    }
  }
  const T* xr = tin + base;
  const T* xi = xr + oplane;
  T* yr = tout + base;
  T* yi = yr + oplane;
  double* pr = psi1 + base;
  double* pim = pr + oplane;
  const T* v = vtot + (long)rep * Ng;
  const T* cre = coef + (long)cre_col * np;
  const T* cim = coef + (long)cim_col * np;
  const long gxy = (long)iy * nx + ix;
  T qr[2 * R + 1], qi[2 * R + 1];
#pragma unroll
  for (int k = 0; k < 2 * R; ++k) {   // planes z0 - R .. z0 + R - 1 of the column
    const int z = z0 - R + k;
    const bool okz = in_xy && z >= 0 && z < nz;
    qr[k] = okz ? xr[(long)z * plane + gxy] : (T)0;
    qi[k] = okz ? xi[(long)z * plane + gxy] : (T)0;
  }
  T nr_next, ni_next;   // plane z + R, loaded one iteration ahead
  {
    const int z = z0 + R;
    const bool okz = in_xy && z < nz;
    nr_next = okz ? xr[(long)z * plane + gxy] : (T)0;
    ni_next = okz ? xi[(long)z * plane + gxy] : (T)0;
  }
  // the point's psi_1, potential and KB list range, loaded one plane ahead
  double p1r = 0.0, p1i = 0.0;
  T vv = (T)0;
  int kb0 = 0, kb1 = 0;
  if (in_xy) {
    const long g = (long)z0 * plane + gxy;
    p1r = pr[g];
    p1i = pim[g];
    vv = v[g];
    if (kb_row) {
      kb0 = kb_row[g];
      kb1 = kb_row[g + 1];
    }
  }
  __syncthreads();   // barriers initialised before anyone waits
  const int lx = tx + kGtXO, ly = ty + R;
  T emax = (T)0;
  bool ok = true;
  int i = 0;
  for (; i < nzb; ++i) {
    qr[2 * R] = nr_next;
    qi[2 * R] = ni_next;
    const double c_p1r = p1r, c_p1i = p1i;
    const T c_vv = vv;
    const int c_kb0 = kb0, c_kb1 = kb1;
    {   // next plane's column value and point data
      const int z = z0 + i + R + 1;
      const bool okz = in_xy && z < nz;
      nr_next = okz ? xr[(long)z * plane + gxy] : (T)0;
      ni_next = okz ? xi[(long)z * plane + gxy] : (T)0;
      if (in_xy && i + 1 < nzb) {
        const long g = (long)(z0 + i + 1) * plane + gxy;
        p1r = pr[g];
        p1i = pim[g];
        vv = v[g];
        if (kb_row) {
          kb0 = kb_row[g];
          kb1 = kb_row[g + 1];
        }
      }
    }
    if (!tc::mbar_wait(&full[i % kGtS], (i / kGtS) & 1)) ok = false;
    const T* tr = tiles + (size_t)(i % kGtS) * 2 * TE;
    const T* ti = tr + TE;
    if (in_xy && ok) {
      const long g = (long)(z0 + i) * plane + gxy;
      T ar = kc.c0 * qr[R], ai = kc.c0 * qi[R];
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const T sr = (tr[ly * TW + lx + m] + tr[ly * TW + lx - m]) +
                     (tr[(ly + m) * TW + lx] + tr[(ly - m) * TW + lx]) + (qr[R + m] + qr[R - m]);
        const T si = (ti[ly * TW + lx + m] + ti[ly * TW + lx - m]) +
                     (ti[(ly + m) * TW + lx] + ti[(ly - m) * TW + lx]) + (qi[R + m] + qi[R - m]);
        ar = fma(kc.cm[m], sr, ar);
        ai = fma(kc.cm[m], si, ai);
      }
      ar = fma(c_vv, qr[R], ar);
      ai = fma(c_vv, qi[R], ai);
      if (c_kb1 > c_kb0) {
        T kr = (T)0, ki = (T)0;
        for (int e = c_kb0; e < c_kb1; ++e) {
          const int p = kb_p[e];
          const T w = kb_w[e];
          kr = fma(w, cre[p], kr);
          ki = fma(w, cim[p], ki);
        }
        ar += kr;
        ai += ki;
      }
      const T nr = kc.c * ai, ni = -kc.c * ar;   // -i c (ar + i ai)
      yr[g] = nr;
      yi[g] = ni;
      pr[g] = c_p1r + (double)nr;
      pim[g] = c_p1i + (double)ni;
      emax = fmax(emax, nr * nr + ni * ni);   // in the terms' precision (a stopping test)
    }
    // every thread is done with slot i % kGtS (or a wait gave up)
    if (__syncthreads_or(!ok)) break;
    if (tid == 0 && i + kGtS < nzb) {   // refill the slot with plane i + kGtS
      const int j = i + kGtS;
      T* dst = tiles + (size_t)(j % kGtS) * 2 * TE;
      const uint32_t bar = tc::saddr(&full[j % kGtS]);
      tc::mbar_expect_tx(bar, kBytes);
      tc::tma_load_4d(tc::saddr(dst), &tm_in, xs, ys, z0 + j, cre_col, bar);
      tc::tma_load_4d(tc::saddr(dst + TE), &tm_in, xs, ys, z0 + j, cim_col, bar);
    }
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) {
      qr[k] = qr[k + 1];
      qi[k] = qi[k + 1];
    }
  }
  if (i < nzb) {   // gave up: wait (bounded) for every issued copy, then leave
    if (tid == 0) {
      atomicCAS(status, 0, (int)RMGTD_ETIMEOUT);
      // the last copy of each slot (older planes' phases are past: waiting on their
      // parity would only run out the limit)
      const int issued = min(nzb, i + kGtS);
      for (int w = max(0, issued - kGtS); w < issued; ++w)
        tc::mbar_wait(&full[w % kGtS], (w / kGtS) & 1);
    }
    return;
  }
  const double bm = block_max((double)emax, sh);
  if (tid == 0) atomic_max_nonneg(&errbits[rep], bm);
}

// The float32 term with two neighbouring x points per thread (vector shared loads): a block of
// 32 x BY threads covers 64 x BY points; the tiles are (64 + 16) x (BY + 12) floats from
// (x0 - 8, y0 - 6).  The x-neighbours of the pair come from 7 float2 loads of its row, the
// y-neighbours from 12 float2 loads, the z-column is a register array of float2 pairs; psi_1
// and the series' float32 pair (hi, lo) move as float2, as do V and the term.  Rows must be a
// whole number of 16-byte units (nx % 4 == 0), so a pair is inside or outside the grid
// together.  No float64 arithmetic: the KB lists and projections are float32 too.  No block
// barrier per plane: each warp arrives on the slot's `empty` mbarrier when done with it, and
// thread 0 refills the slot once all have (the warps run up to kG2S planes apart).
constexpr int kG2X = 64;   // points per block along x
constexpr int kG2S = 4;    // planes in flight
constexpr int kG2Z = 12;   // z-planes per block, about

template <int BY>
__host__ __device__ constexpr int gt2_tile_elems() {
  return (BY + 2 * kFdRadius) * (kG2X + 2 * kGtXO);
}

template <int BY>
__host__ __device__ constexpr size_t gt2_smem_bytes() {
  return sizeof(float) * 2 * gt2_tile_elems<BY>() * kG2S + 2 * sizeof(uint64_t) * kG2S + 1024;
}

template <int BY>
__global__ void __launch_bounds__(32 * BY)
k_gp_term_tma2(const __grid_constant__ CUtensorMap tm_in, const float* __restrict__ tin,
               float* __restrict__ tout, float* __restrict__ acc, long lo_off, int first,
               const float* __restrict__ vtot, const int* __restrict__ kb_row,
               const int* __restrict__ kb_p, const float* __restrict__ kb_w,
               const float* __restrict__ coef, int np, int nocc,
               int nx, int ny, int nz, int zchunk, int nzc, const GpTermCoef<float> kc,
               const int* __restrict__ sact, unsigned long long* __restrict__ errbits,
               int* __restrict__ status) {
  constexpr int R = kFdRadius;
  constexpr int TW = kG2X + 2 * kGtXO;
  constexpr int TE = gt2_tile_elems<BY>();
  constexpr uint32_t kBytes = 2u * TE * sizeof(float);
  extern __shared__ unsigned char gt2_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(gt2_raw) + 1023) & ~(uintptr_t)1023);
  float* tiles = reinterpret_cast<float*>(smem);   // [kG2S][2][BY + 2R][TW]
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + sizeof(float) * 2 * TE * kG2S);
  uint64_t* empty = full + kG2S;   // all warps done with a slot (one arrival per warp)
  __shared__ double sh[32];
  const int col = blockIdx.z / nzc;
  const int rep = col / nocc, n = col - rep * nocc;
  if (!sact[rep]) return;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int z0 = (blockIdx.z % nzc) * zchunk, z1 = min(nz, z0 + zchunk), nzb = z1 - z0;
  const int ix = blockIdx.x * kG2X + 2 * tx, iy = blockIdx.y * BY + ty;
  const bool in_xy = ix < nx && iy < ny;   // ix even, nx % 4 == 0: ix + 1 < nx too
  const long plane = (long)nx * ny, Ng = plane * nz, oplane = (long)nocc * Ng;
  const long base = (long)rep * 2 * oplane + (long)n * Ng;
  const int cre_col = rep * 2 * nocc + n, cim_col = cre_col + nocc;
  const int xs = blockIdx.x * kG2X - kGtXO, ys = blockIdx.y * BY - R;
  if (tid == 0) {
    for (int s = 0; s < kG2S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], BY);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int i = 0; i < min(kG2S, nzb); ++i) {
      float* dst = tiles + (size_t)i * 2 * TE;
      const uint32_t bar = tc::saddr(&full[i]);
      tc::mbar_expect_tx(bar, kBytes);
      tc::tma_load_4d(tc::saddr(dst), &tm_in, xs, ys, z0 + i, cre_col, bar);
      tc::tma_load_4d(tc::saddr(dst + TE), &tm_in, xs, ys, z0 + i, cim_col, bar);
    }
  }
  const float* xr = tin + base;
  const float* xi = xr + oplane;
  float* yr = tout + base;
  float* yi = yr + oplane;
  float* hr = acc + base;          // the sum's hi and lo, real and imaginary
  float* hi_ = hr + oplane;
  float* lr = hr + lo_off;
  float* li = hi_ + lo_off;
  const float* v = vtot + (long)rep * Ng;
  const float* cre = coef + (long)cre_col * np;
  const float* cim = coef + (long)cim_col * np;
  const long gxy = (long)iy * nx + ix;
  float2 qr[2 * R + 1], qi[2 * R + 1];
#pragma unroll
  for (int k = 0; k < 2 * R; ++k) {
    const int z = z0 - R + k;
    const bool okz = in_xy && z >= 0 && z < nz;
    qr[k] = okz ? *reinterpret_cast<const float2*>(xr + (long)z * plane + gxy) : make_float2(0.f, 0.f);
    qi[k] = okz ? *reinterpret_cast<const float2*>(xi + (long)z * plane + gxy) : make_float2(0.f, 0.f);
  }
  float2 nr_next, ni_next;
  {
    const int z = z0 + R;
    const bool okz = in_xy && z < nz;
    nr_next = okz ? *reinterpret_cast<const float2*>(xr + (long)z * plane + gxy) : make_float2(0.f, 0.f);
    ni_next = okz ? *reinterpret_cast<const float2*>(xi + (long)z * plane + gxy) : make_float2(0.f, 0.f);
  }
  const float2 zero2 = make_float2(0.f, 0.f);
  float2 ahr = zero2, ahi = zero2, alr = zero2, ali = zero2;   // the sum, one plane ahead
  float2 vv = zero2;
  int kb0 = 0, kb1 = 0, kb2 = 0;
  if (in_xy) {
    const long g = (long)z0 * plane + gxy;
    if (!first) {
      ahr = *reinterpret_cast<const float2*>(hr + g);
      ahi = *reinterpret_cast<const float2*>(hi_ + g);
      alr = *reinterpret_cast<const float2*>(lr + g);
      ali = *reinterpret_cast<const float2*>(li + g);
    }
    vv = *reinterpret_cast<const float2*>(v + g);
    if (kb_row) {
      kb0 = kb_row[g];
      kb1 = kb_row[g + 1];
      kb2 = kb_row[g + 2];
    }
  }
  __syncthreads();
  const int lx = 2 * tx + kGtXO, ly = ty + R;
  float emax = 0.f;
  bool ok = true;
  int issued = min(kG2S, nzb);   // planes whose copies thread 0 issued
  for (int i = 0; i < nzb; ++i) {
    qr[2 * R] = nr_next;
    qi[2 * R] = ni_next;
    const float2 c_ahr = ahr, c_ahi = ahi, c_alr = alr, c_ali = ali;
    const float2 c_vv = vv;
    const int c_kb0 = kb0, c_kb1 = kb1, c_kb2 = kb2;
    {
      const int z = z0 + i + R + 1;
      const bool okz = in_xy && z < nz;
      nr_next = okz ? *reinterpret_cast<const float2*>(xr + (long)z * plane + gxy) : zero2;
      ni_next = okz ? *reinterpret_cast<const float2*>(xi + (long)z * plane + gxy) : zero2;
      if (in_xy && i + 1 < nzb) {
        const long g = (long)(z0 + i + 1) * plane + gxy;
        if (!first) {
          ahr = *reinterpret_cast<const float2*>(hr + g);
          ahi = *reinterpret_cast<const float2*>(hi_ + g);
          alr = *reinterpret_cast<const float2*>(lr + g);
          ali = *reinterpret_cast<const float2*>(li + g);
        }
        vv = *reinterpret_cast<const float2*>(v + g);
        if (kb_row) {
          kb0 = kb_row[g];
          kb1 = kb_row[g + 1];
          kb2 = kb_row[g + 2];
        }
      }
    }
    if (ok && !tc::mbar_wait(&full[i % kG2S], (i / kG2S) & 1)) ok = false;
    const float* tr = tiles + (size_t)(i % kG2S) * 2 * TE;
    const float* ti = tr + TE;
    if (in_xy && ok) {
      const long g = (long)(z0 + i) * plane + gxy;
      // the row segment lx - 6 .. lx + 7 of both planes (7 float2 each)
      float xr14[14], xi14[14];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const float2 a = *reinterpret_cast<const float2*>(tr + ly * TW + lx - R + 2 * k);
        const float2 b = *reinterpret_cast<const float2*>(ti + ly * TW + lx - R + 2 * k);
        xr14[2 * k] = a.x;
        xr14[2 * k + 1] = a.y;
        xi14[2 * k] = b.x;
        xi14[2 * k + 1] = b.y;
      }
      // point 0 at xr14[R], point 1 at xr14[R + 1]
      float ar0 = kc.c0 * qr[R].x, ar1 = kc.c0 * qr[R].y, ai0 = kc.c0 * qi[R].x, ai1 = kc.c0 * qi[R].y;
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        const float2 ur = *reinterpret_cast<const float2*>(tr + (ly + m) * TW + lx);
        const float2 dr = *reinterpret_cast<const float2*>(tr + (ly - m) * TW + lx);
        const float2 ui = *reinterpret_cast<const float2*>(ti + (ly + m) * TW + lx);
        const float2 di = *reinterpret_cast<const float2*>(ti + (ly - m) * TW + lx);
        const float sr0 = (xr14[R + m] + xr14[R - m]) + (ur.x + dr.x) + (qr[R + m].x + qr[R - m].x);
        const float sr1 = (xr14[R + 1 + m] + xr14[R + 1 - m]) + (ur.y + dr.y) + (qr[R + m].y + qr[R - m].y);
        const float si0 = (xi14[R + m] + xi14[R - m]) + (ui.x + di.x) + (qi[R + m].x + qi[R - m].x);
        const float si1 = (xi14[R + 1 + m] + xi14[R + 1 - m]) + (ui.y + di.y) + (qi[R + m].y + qi[R - m].y);
        ar0 = fmaf(kc.cm[m], sr0, ar0);
        ar1 = fmaf(kc.cm[m], sr1, ar1);
        ai0 = fmaf(kc.cm[m], si0, ai0);
        ai1 = fmaf(kc.cm[m], si1, ai1);
      }
      ar0 = fmaf(c_vv.x, qr[R].x, ar0);
      ar1 = fmaf(c_vv.y, qr[R].y, ar1);
      ai0 = fmaf(c_vv.x, qi[R].x, ai0);
      ai1 = fmaf(c_vv.y, qi[R].y, ai1);
      if (c_kb2 > c_kb0) {
        float kr0 = 0.f, ki0 = 0.f, kr1 = 0.f, ki1 = 0.f;
        for (int e = c_kb0; e < c_kb1; ++e) {
          const int p = kb_p[e];
          const float w = kb_w[e];
          kr0 = fmaf(w, cre[p], kr0);
          ki0 = fmaf(w, cim[p], ki0);
        }
        for (int e = c_kb1; e < c_kb2; ++e) {
          const int p = kb_p[e];
          const float w = kb_w[e];
          kr1 = fmaf(w, cre[p], kr1);
          ki1 = fmaf(w, cim[p], ki1);
        }
        ar0 += kr0;
        ai0 += ki0;
        ar1 += kr1;
        ai1 += ki1;
      }
      const float2 nr = make_float2(kc.c * ai0, kc.c * ai1), ni = make_float2(-kc.c * ar0, -kc.c * ar1);
      *reinterpret_cast<float2*>(yr + g) = nr;
      *reinterpret_cast<float2*>(yi + g) = ni;
      if (first) {
        *reinterpret_cast<float2*>(hr + g) = nr;
        *reinterpret_cast<float2*>(hi_ + g) = ni;
        *reinterpret_cast<float2*>(lr + g) = zero2;
        *reinterpret_cast<float2*>(li + g) = zero2;
      } else {
        float2 sr, si, er, ei;
        two_sum(c_ahr.x, nr.x, sr.x, er.x);
        two_sum(c_ahr.y, nr.y, sr.y, er.y);
        two_sum(c_ahi.x, ni.x, si.x, ei.x);
        two_sum(c_ahi.y, ni.y, si.y, ei.y);
        *reinterpret_cast<float2*>(hr + g) = sr;
        *reinterpret_cast<float2*>(hi_ + g) = si;
        *reinterpret_cast<float2*>(lr + g) = make_float2(c_alr.x + er.x, c_alr.y + er.y);
        *reinterpret_cast<float2*>(li + g) = make_float2(c_ali.x + ei.x, c_ali.y + ei.y);
      }
      emax = fmaxf(emax, fmaxf(nr.x * nr.x + ni.x * ni.x, nr.y * nr.y + ni.y * ni.y));
    }
    // this warp is done with slot i % kG2S; thread 0 refills it once every warp is
    // (no block barrier: the warps run up to kG2S planes apart)
    __syncwarp();
    if ((tid & 31) == 0) tc::mbar_arrive(&empty[i % kG2S]);
    if (tid == 0 && i + kG2S < nzb && ok) {
      if (!tc::mbar_wait(&empty[i % kG2S], (i / kG2S) & 1)) {
        ok = false;
      } else {
        const int j = i + kG2S;
        float* dst = tiles + (size_t)(j % kG2S) * 2 * TE;
        const uint32_t bar = tc::saddr(&full[j % kG2S]);
        tc::mbar_expect_tx(bar, kBytes);
        tc::tma_load_4d(tc::saddr(dst), &tm_in, xs, ys, z0 + j, cre_col, bar);
        tc::tma_load_4d(tc::saddr(dst + TE), &tm_in, xs, ys, z0 + j, cim_col, bar);
        issued = j + 1;
      }
    }
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) {
      qr[k] = qr[k + 1];
      qi[k] = qi[k + 1];
    }
  }
  if (__syncthreads_or(!ok)) {   // a wait gave up: wait (bounded) for the copies in flight
    if (tid == 0) {
      atomicCAS(status, 0, (int)RMGTD_ETIMEOUT);
      for (int w = max(0, issued - kG2S); w < issued; ++w)
        tc::mbar_wait(&full[w % kG2S], (w / kG2S) & 1);
    }
    return;
  }
  const double bm = block_max((double)emax, sh);
  if (tid == 0) atomic_max_nonneg(&errbits[rep], bm);
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

// The first Hartree solve's guess at the start of a step: with a = V_H now (the last solve),
// vh <- 3 a - 3 vh1 + vh2 (two earlier steps known), 2 a - vh1 (one), a (none): V_H one step
// ahead to O(dt^3); then vh2 <- vh1, vh1 <- a.  The guess changes only the iteration count.
__global__ void k_gp_vh_guess(double* __restrict__ vh, double* __restrict__ vh1,
                              double* __restrict__ vh2, int hist, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const double a = vh[e], b = vh1[e];
    vh[e] = hist >= 2 ? 3.0 * (a - b) + vh2[e] : hist == 1 ? 2.0 * a - b : a;
    vh2[e] = b;
    vh1[e] = a;
  }
}

// psi0f = psi in float32 (float32 terms: once per step, the first term's input)
__global__ void k_gp_to_f32(const double* __restrict__ psi, float* __restrict__ out, long n) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    out[e] = (float)psi[e];
}

// float32 terms: rho_r = rho0_r + sum_n f_n (2 Re(conj(psi0_n) s_n) + |s_n|^2), the density of
// psi_1 = psi_0 + s (s = the series' sum hi + lo, taken as hi: |lo| is below hi's rounding)
// as a float32 change on the float64 density of psi_0; no float64 arithmetic per orbital
__global__ void k_gp_drho(const float* __restrict__ psi0f, const float* __restrict__ hi,
                          const float* __restrict__ fs, int nocc, long Ng,
                          const double* __restrict__ rho0, double* __restrict__ rho) {
  const int r = blockIdx.y;
  const long plane = (long)nocc * Ng;
  const float* p = psi0f + 2 * r * plane;
  const float* h = hi + 2 * r * plane;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x) {
    float d = 0.f;
    for (int n = 0; n < nocc; ++n) {
      const long o = (long)n * Ng + g;
      const float pr = p[o], pi = p[plane + o], hr = h[o], hm = h[plane + o];
      d = fmaf(fs[n], fmaf(2.f, fmaf(pr, hr, pi * hm), fmaf(hr, hr, hm * hm)), d);
    }
    rho[r * Ng + g] = rho0[r * Ng + g] + (double)d;
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

// Gram G_nm = sum_g psi_n conj(psi_m) of a few orbitals (n <= m pairs): every block stages
// kZgP points of all orbitals (both planes) in shared memory and each thread accumulates its
// pairs over the block's chunks; per-block partials [block][pair][2], reduced in a fixed order.
constexpr int kZgP = 32, kZgMaxPairsPerThread = 10, kZgThreads = 256;
constexpr int kZgMaxN = 64;   // 2080 pairs <= 256 x 10 and 2 x 64 x 32 doubles of staging

__global__ void __launch_bounds__(kZgThreads)
k_gp_zgram_partial(int nocc, long Ng, const double* __restrict__ re, const double* __restrict__ im,
                   double* __restrict__ part) {
  __shared__ double sr[kZgMaxN][kZgP];
  __shared__ double si[kZgMaxN][kZgP];
  const int npairs = nocc * (nocc + 1) / 2;
  double ar[kZgMaxPairsPerThread], ai[kZgMaxPairsPerThread];
  int pn[kZgMaxPairsPerThread], pm[kZgMaxPairsPerThread];
#pragma unroll
  for (int u = 0; u < kZgMaxPairsPerThread; ++u) {
    ar[u] = ai[u] = 0.0;
    int q = threadIdx.x + u * kZgThreads, n = 0;
    while (q >= nocc - n && n < nocc) {   // pair index -> (n, m), n <= m
      q -= nocc - n;
      ++n;
    }
    pn[u] = n;
    pm[u] = n + q;
  }
  for (long c0 = blockIdx.x * (long)kZgP; c0 < Ng; c0 += (long)gridDim.x * kZgP) {
    __syncthreads();
    for (int e = threadIdx.x; e < nocc * kZgP; e += kZgThreads) {
      const int n = e / kZgP, p = e - n * kZgP;
      const long g = c0 + p;
      sr[n][p] = g < Ng ? re[(long)n * Ng + g] : 0.0;
      si[n][p] = g < Ng ? im[(long)n * Ng + g] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kZgMaxPairsPerThread; ++u) {
      if (threadIdx.x + u * kZgThreads >= npairs) break;
      const int n = pn[u], m = pm[u];
      double xr = ar[u], xi = ai[u];
      for (int p = 0; p < kZgP; ++p) {
        xr = fma(sr[n][p], sr[m][p], fma(si[n][p], si[m][p], xr));
        xi = fma(si[n][p], sr[m][p], -fma(sr[n][p], si[m][p], -xi));
      }
      ar[u] = xr;
      ai[u] = xi;
    }
  }
#pragma unroll
  for (int u = 0; u < kZgMaxPairsPerThread; ++u) {
    const int q = threadIdx.x + u * kZgThreads;
    if (q >= npairs) break;
    part[((long)blockIdx.x * npairs + q) * 2] = ar[u];
    part[((long)blockIdx.x * npairs + q) * 2 + 1] = ai[u];
  }
}

// G = scale * sum over blocks (fixed order), full Hermitian (gre, gim) from the n <= m pairs
// one warp per pair (the lanes stride over the block partials, then a warp sum: a serial
// loop over hundreds of partials per thread was latency-bound)
__global__ void k_gp_zgram_reduce(int nocc, int nblk, const double* __restrict__ part, double scale,
                                  double* __restrict__ gre, double* __restrict__ gim) {
  const int npairs = nocc * (nocc + 1) / 2;
  const int lane = threadIdx.x & 31, nwarp = (gridDim.x * blockDim.x) >> 5;
  for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < npairs; q += nwarp) {
    int n = 0, r = q;
    while (r >= nocc - n) {
      r -= nocc - n;
      ++n;
    }
    const int m = n + r;
    double xr = 0.0, xi = 0.0;
    for (int b = lane; b < nblk; b += 32) {
      xr += part[((long)b * npairs + q) * 2];
      xi += part[((long)b * npairs + q) * 2 + 1];
    }
    xr = warp_sum(xr);
    xi = warp_sum(xi);
    if (lane == 0) {
      gre[(long)n * nocc + m] = scale * xr;
      gim[(long)n * nocc + m] = scale * xi;
      gre[(long)m * nocc + n] = scale * xr;
      gim[(long)m * nocc + n] = -scale * xi;
    }
  }
}

// X = L^-1 of the complex lower Cholesky factor (one block; thread j solves L x = e_j)
__global__ void k_ztri_inverse(int N, const double* __restrict__ lre, const double* __restrict__ lim,
                               double* __restrict__ xre, double* __restrict__ xim) {
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    for (int i = 0; i < j; ++i) {
      xre[(long)i * N + j] = 0.0;
      xim[(long)i * N + j] = 0.0;
    }
    for (int i = j; i < N; ++i) {
      double sr = (i == j) ? 1.0 : 0.0, si = 0.0;
      for (int k = j; k < i; ++k) {
        const double ar = lre[(long)i * N + k], ai = lim[(long)i * N + k];
        const double br = xre[(long)k * N + j], bi = xim[(long)k * N + j];
        sr -= ar * br - ai * bi;
        si -= ar * bi + ai * br;
      }
      const double d = lre[(long)i * N + i];   // real positive pivot
      xre[(long)i * N + j] = sr / d;
      xim[(long)i * N + j] = si / d;
    }
  }
}

// psi_out_n = sum_{m <= n} X_nm psi_in_m per grid point, the point's orbitals in registers.
// X = L^-1 is the identity up to the series' departure from unitarity, so when every entry of
// X - I is below kXSmall the kernel forms psi_out = psi_in + (X - I) psi_in with the correction
// in float32 (its rounding, ~1e-7 of a correction below 1e-6 of |psi|, stays under 1e-13 of
// |psi|): per orbital two conversions and one float64 add instead of 2(n + 1) complex float64
// multiply-adds.  Otherwise the product is float64 throughout.
constexpr double kXSmall = 1e-6;

template <int MAXN>
__global__ void __launch_bounds__(256)
k_gp_xapply(int nocc, long Ng, const double* __restrict__ xre, const double* __restrict__ xim,
            const double* __restrict__ in, double* __restrict__ out) {
  __shared__ double sxr[MAXN * MAXN], sxi[MAXN * MAXN];
  __shared__ float sfr[MAXN * MAXN], sfi[MAXN * MAXN];
  bool big = false;
  for (int e = threadIdx.x; e < nocc * nocc; e += blockDim.x) {
    const int n = e / nocc, m = e - n * nocc;
    const double dr = xre[e] - (n == m ? 1.0 : 0.0), di = xim[e];
    sxr[e] = xre[e];
    sxi[e] = di;
    sfr[e] = (float)dr;
    sfi[e] = (float)di;
    big = big || !(fabs(dr) <= kXSmall && fabs(di) <= kXSmall);
  }
  big = __syncthreads_or(big);   // uniform over the block
  const long plane = (long)nocc * Ng;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng; g += (long)gridDim.x * blockDim.x) {
    double yr[MAXN], yi[MAXN];
#pragma unroll
    for (int m = 0; m < MAXN; ++m) {
      yr[m] = m < nocc ? in[(long)m * Ng + g] : 0.0;
      yi[m] = m < nocc ? in[plane + (long)m * Ng + g] : 0.0;
    }
    if (!big) {
      float fr[MAXN], fi[MAXN];
#pragma unroll
      for (int m = 0; m < MAXN; ++m) {
        fr[m] = (float)yr[m];
        fi[m] = (float)yi[m];
      }
#pragma unroll
      for (int n = 0; n < MAXN; ++n) {
        if (n >= nocc) break;
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int m = 0; m <= n; ++m) {
          const float ar = sfr[n * nocc + m], ai = sfi[n * nocc + m];
          sr = fmaf(ar, fr[m], fmaf(-ai, fi[m], sr));
          si = fmaf(ar, fi[m], fmaf(ai, fr[m], si));
        }
        out[(long)n * Ng + g] = yr[n] + (double)sr;
        out[plane + (long)n * Ng + g] = yi[n] + (double)si;
      }
      continue;
    }
#pragma unroll
    for (int n = 0; n < MAXN; ++n) {
      if (n >= nocc) break;
      double sr = 0.0, si = 0.0;
#pragma unroll
      for (int m = 0; m <= n; ++m) {
        const double ar = sxr[n * nocc + m], ai = sxi[n * nocc + m];
        sr = fma(ar, yr[m], fma(-ai, yi[m], sr));
        si = fma(ar, yi[m], fma(ai, yr[m], si));
      }
      out[(long)n * Ng + g] = sr;
      out[plane + (long)n * Ng + g] = si;
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

constexpr int kGpBX = 32, kGpBY = 8, kGpZ = 16, kGtZ = 32;

// tensor maps of the term buffers (and of psi0f) for the TMA kernel: 4-D {nx, ny, nz, columns}, box
// {BX + 16, BY + 12, 1, 1}, zero fill outside; only when a row of x is a whole number of
// 16-byte units (then every stride is)
template <typename T>
bool gp_encode_term_maps(rmgtd_ctx* ctx) {
  const EncodeTiledFn f = tensor_map_encoder();
  if (!f || ((long)ctx->nx * sizeof(T)) % 16 != 0) return false;
  cudaError_t e;
  if constexpr (sizeof(T) == sizeof(float))   // the two-point float32 kernel: 64-wide tiles
    e = cudaFuncSetAttribute(k_gp_term_tma2<kGpBY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gt2_smem_bytes<kGpBY>());
  else
    e = cudaFuncSetAttribute(k_gp_term_tma<T, kGpBX, kGpBY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gt_smem_bytes<T, kGpBX, kGpBY>());
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int bx = sizeof(T) == sizeof(float) ? kG2X : kGpBX;
  const cuuint64_t cols = 2ull * ctx->N * ctx->nrep;
  const cuuint64_t dims[4] = {(cuuint64_t)ctx->nx, (cuuint64_t)ctx->ny, (cuuint64_t)ctx->nz, cols};
  const cuuint64_t strides[3] = {(cuuint64_t)ctx->nx * sizeof(T),
                                 (cuuint64_t)ctx->nx * ctx->ny * sizeof(T),
                                 (cuuint64_t)ctx->Ng * sizeof(T)};
  const cuuint32_t box[4] = {(cuuint32_t)(bx + 2 * kGtXO), (cuuint32_t)(kGpBY + 2 * kFdRadius), 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt =
      sizeof(T) == sizeof(double) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  for (int b = 0; b < (ctx->gp_psi0f ? 3 : 2); ++b) {
    void* base = b == 0 ? ctx->gp_ta : b == 1 ? ctx->gp_tb : (void*)ctx->gp_psi0f;
    void* map = b == 0 ? (void*)ctx->gp_tm_a : b == 1 ? (void*)ctx->gp_tm_b : (void*)ctx->gp_tm_0;
    if (f(reinterpret_cast<CUtensorMap*>(map), dt, 4, base, dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

int gp_zgram_blocks(rmgtd_ctx* ctx) {
  return (int)std::max<long>(1, std::min<long>(ceil_div(ctx->Ng, kZgP), 4L * ctx->num_sms));
}

// the mixed path's series terms are float32
bool gp_f32(const rmgtd_ctx* ctx) { return ctx->opt.precision == RMGTD_PREC_MIXED; }

// one series term for every replica whose series is running: tout = (-i dt/k) Hbar tin,
// psi_1 += tout, errbits <- max|tout|^2 (the KB projections of tin first)
template <typename T>
int gp_term(rmgtd_ctx* ctx, const T* tin, T* tout, double c, bool first) {
  const int N = ctx->N, nrep = ctx->nrep;
  if (ctx->nproj > 0) {   // one block per projector and group of real columns
    const int ncols = 2 * N * nrep;
    k_gp_kb_project<T><<<dim3(ctx->nproj, ceil_div(ncols, kKbCols)), kKbThreads, 0, ctx->stream>>>(
        tin, ctx->Ng, ncols, 2 * N, ctx->gp_sact, ctx->poff, ctx->gp_kb_pt, (const T*)ctx->gp_pv,
        ctx->h3, (T*)ctx->gp_coef);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_kb_project");
  }
  const T* kb_w = (const T*)ctx->gp_kb_w;
  const T* coef = (const T*)ctx->gp_coef;
  const long lo_off = 2L * N * ctx->Ng * nrep;
  const GpTermCoef<T> kc = gp_term_coef<T>(ctx->h, c);
  T* acc;
  if constexpr (sizeof(T) == sizeof(float)) acc = ctx->gp_acc;
  else acc = ctx->gp_psi1;
  if (ctx->gp_tma) {   // x-y tiles by TMA from the term's tensor map
    const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(
        (const void*)tin == ctx->gp_ta ? ctx->gp_tm_a
        : (const void*)tin == ctx->gp_tb ? ctx->gp_tm_b : ctx->gp_tm_0);
    if constexpr (sizeof(T) == sizeof(float)) {
      // z split evenly into chunks of about kG2Z planes (more, shorter blocks fill the SMs'
      // two block slots better than 32-plane chunks: 16.0 vs 17.0 ms per step on the ring)
      const int nzc = ceil_div(ctx->nz, kG2Z), zc = ceil_div(ctx->nz, nzc);
      const dim3 grid(ceil_div(ctx->nx, kG2X), ceil_div(ctx->ny, kGpBY), nrep * N * nzc);
      k_gp_term_tma2<kGpBY><<<grid, dim3(32, kGpBY), gt2_smem_bytes<kGpBY>(), ctx->stream>>>(
          *tm, tin, tout, acc, lo_off, first ? 1 : 0, (const float*)ctx->gp_vtot, ctx->gp_kb_row,
          ctx->gp_kb_p, kb_w, coef, ctx->nproj, N, ctx->nx, ctx->ny, ctx->nz, zc, nzc,
          kc, ctx->gp_sact, ctx->errbits, ctx->status);
      ++ctx->launches;
      RMGTD_LAUNCH(ctx, "k_gp_term_tma2");
    } else {
      const int nzc = ceil_div(ctx->nz, kGtZ);
      const dim3 grid(ceil_div(ctx->nx, kGpBX), ceil_div(ctx->ny, kGpBY), nrep * N * nzc);
      k_gp_term_tma<T, kGpBX, kGpBY><<<grid, dim3(kGpBX, kGpBY), gt_smem_bytes<T, kGpBX, kGpBY>(),
                                        ctx->stream>>>(
          *tm, tin, tout, acc, (const T*)ctx->gp_vtot, ctx->gp_kb_row, ctx->gp_kb_p,
          kb_w, coef, ctx->nproj, N, ctx->nx, ctx->ny, ctx->nz, kGtZ, nzc,
          kc, ctx->gp_sact, ctx->errbits, ctx->status);
      ++ctx->launches;
      RMGTD_LAUNCH(ctx, "k_gp_term_tma");
    }
    return RMGTD_OK;
  }
  const int nzc = ceil_div(ctx->nz, kGpZ);
  const dim3 grid(ceil_div(ctx->nx, kGpBX), ceil_div(ctx->ny, kGpBY), nrep * N * nzc);
  k_gp_term_fused<T, kGpBX, kGpBY><<<grid, dim3(kGpBX, kGpBY), 0, ctx->stream>>>(
      tin, tout, acc, lo_off, first ? 1 : 0, (const T*)ctx->gp_vtot, ctx->gp_kb_row,
      ctx->gp_kb_p, kb_w, coef, ctx->nproj, N, ctx->nx, ctx->ny, ctx->nz, kGpZ, nzc,
      kc, ctx->gp_sact, ctx->errbits);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_term_fused");
  return RMGTD_OK;
}

// KB lists by grid point (CSR) from the projector boxes: entry (p, E_p beta_p(r)) for every
// projector whose box holds the point; the grid index of every box entry; weights and box
// values in the terms' precision
template <typename T>
int gp_build_kb_lists(rmgtd_ctx* ctx) {
  const int np = ctx->nproj;
  const long Ng = ctx->Ng;
  const long long nval = ctx->h_poff[np];
  std::vector<double> val(nval);
  RMGTD_CUDA(ctx, cudaMemcpy(val.data(), ctx->pval, sizeof(double) * nval, cudaMemcpyDeviceToHost));
  std::vector<int> cnt(Ng + 1, 0);
  auto point = [&](int p, long long e) {
    const int* b = &ctx->h_pbox[6 * p];
    const long long bxy = (long long)b[3] * b[4];
    const long long z = b[2] + e / bxy, y = b[1] + (e / b[3]) % b[4], x = b[0] + e % b[3];
    return (long)((z * ctx->ny + y) * ctx->nx + x);
  };
  for (int p = 0; p < np; ++p)
    for (long long e = 0; e < ctx->h_poff[p + 1] - ctx->h_poff[p]; ++e) ++cnt[point(p, e) + 1];
  for (long g = 0; g < Ng; ++g) cnt[g + 1] += cnt[g];
  if ((long long)cnt[Ng] != nval) return set_error(ctx, RMGTD_EINVAL, "KB lists: box count mismatch");
  std::vector<int> pos(cnt.begin(), cnt.end() - 1), pidx(nval), pt(nval);
  std::vector<T> w(nval), pv(nval);
  for (int p = 0; p < np; ++p)
    for (long long e = 0; e < ctx->h_poff[p + 1] - ctx->h_poff[p]; ++e) {
      const long g = point(p, e);
      const int k = pos[g]++;
      pidx[k] = p;
      w[k] = (T)(ctx->h_Ekb[p] * val[ctx->h_poff[p] + e]);
      pt[ctx->h_poff[p] + e] = (int)g;
      pv[ctx->h_poff[p] + e] = (T)val[ctx->h_poff[p] + e];
    }
  const size_t n1 = std::max<long long>(nval, 1);
  ctx->gp_kb_row = (int*)dev_alloc(ctx, sizeof(int) * (Ng + 1));
  ctx->gp_kb_p = (int*)dev_alloc(ctx, sizeof(int) * n1);
  ctx->gp_kb_w = dev_alloc(ctx, sizeof(T) * n1);
  ctx->gp_kb_pt = (int*)dev_alloc(ctx, sizeof(int) * n1);
  ctx->gp_pv = dev_alloc(ctx, sizeof(T) * n1);
  if (!ctx->gp_kb_row || !ctx->gp_kb_p || !ctx->gp_kb_w || !ctx->gp_kb_pt || !ctx->gp_pv)
    return set_error(ctx, RMGTD_ENOMEM, "KB lists");
  RMGTD_CUDA(ctx, cudaMemcpy(ctx->gp_kb_row, cnt.data(), sizeof(int) * (Ng + 1), cudaMemcpyHostToDevice));
  RMGTD_CUDA(ctx, cudaMemcpy(ctx->gp_kb_p, pidx.data(), sizeof(int) * nval, cudaMemcpyHostToDevice));
  RMGTD_CUDA(ctx, cudaMemcpy(ctx->gp_kb_w, w.data(), sizeof(T) * nval, cudaMemcpyHostToDevice));
  RMGTD_CUDA(ctx, cudaMemcpy(ctx->gp_kb_pt, pt.data(), sizeof(int) * nval, cudaMemcpyHostToDevice));
  RMGTD_CUDA(ctx, cudaMemcpy(ctx->gp_pv, pv.data(), sizeof(T) * nval, cudaMemcpyHostToDevice));
  return RMGTD_OK;
}

}  // namespace

int gridprop_setup(rmgtd_ctx* ctx) {
  const int nocc = ctx->N, nrep = ctx->nrep;
  const long Ng = ctx->Ng, plane = (long)nocc * Ng;
  // the term kernels take one block row per replica, orbital and z chunk (at least
  // ceil(nz / kG2Z) chunks): the launch grid's z extent is at most 65535
  if ((long)nrep * nocc * ceil_div(ctx->nz, std::min(kG2Z, kGpZ)) > 65535L)
    return set_error(ctx, RMGTD_EINVAL,
                     "grid_basis: replicas x orbitals x z chunks exceed the launch grid (65535)");
  const size_t psz = sizeof(double) * 2 * plane * nrep;
  const size_t tsz = gp_f32(ctx) ? sizeof(float) : sizeof(double);
  ctx->gp_psi = (double*)dev_alloc(ctx, psz);
  ctx->gp_psi1 = (double*)dev_alloc(ctx, psz);
  ctx->gp_ht = (double*)dev_alloc(ctx, psz);
  ctx->gp_ta = dev_alloc(ctx, tsz * 2 * plane * nrep);
  ctx->gp_tb = dev_alloc(ctx, tsz * 2 * plane * nrep);
  const size_t vsz = sizeof(double) * Ng * nrep;
  ctx->gp_v0 = (double*)dev_alloc(ctx, vsz);
  ctx->gp_vm1 = (double*)dev_alloc(ctx, vsz);
  if (ctx->opt.seed_order == 2) {
    ctx->gp_vm2 = (double*)dev_alloc(ctx, vsz);
    if (!ctx->gp_vm2) return set_error(ctx, RMGTD_ENOMEM, "grid propagation buffers");
  }
  ctx->gp_v1 = (double*)dev_alloc(ctx, vsz);
  ctx->gp_vtot = dev_alloc(ctx, tsz * Ng * nrep);
  ctx->gp_ebar = (double*)dev_alloc(ctx, sizeof(double) * 3 * nrep);
  ctx->gp_active = (int*)dev_alloc(ctx, sizeof(int) * nrep);
  ctx->gp_sact = (int*)dev_alloc(ctx, sizeof(int) * 3 * nrep);
  ctx->gp_coef = dev_alloc(ctx, tsz * std::max(ctx->nproj, 1) * 2L * nocc * nrep);
  if (ctx->hartree_xc) {
    ctx->gp_vh1 = (double*)dev_alloc(ctx, vsz);
    ctx->gp_vh2 = (double*)dev_alloc(ctx, vsz);
    if (!ctx->gp_vh1 || !ctx->gp_vh2) return set_error(ctx, RMGTD_ENOMEM, "grid propagation buffers");
    ctx->gp_vh_hist = 0;
  }
  if (gp_f32(ctx)) {
    ctx->gp_acc = (float*)ctx->gp_ht;   // hi + lo floats: the size of gp_ht
    ctx->gp_psi0f = (float*)dev_alloc(ctx, sizeof(float) * 2 * plane * nrep);
    ctx->gp_rho0 = (double*)dev_alloc(ctx, sizeof(double) * Ng * nrep);
    ctx->gp_f32occ = (float*)dev_alloc(ctx, sizeof(float) * nocc);
    if (!ctx->gp_psi0f || !ctx->gp_rho0 || !ctx->gp_f32occ)
      return set_error(ctx, RMGTD_ENOMEM, "grid propagation buffers");
    std::vector<float> ff(ctx->f.begin(), ctx->f.begin() + nocc);
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->gp_f32occ, ff.data(), sizeof(float) * nocc, cudaMemcpyHostToDevice));
  }
  ctx->gp_gram = (double*)dev_alloc(ctx, sizeof(double) * 5 * (size_t)nocc * nocc);
  if (nocc <= kZgMaxN)
    ctx->gp_zpart = (double*)dev_alloc(
        ctx, sizeof(double) * 2 * (size_t)gp_zgram_blocks(ctx) * (nocc * (nocc + 1) / 2));
  ctx->gp_obs = (double*)dev_alloc(ctx, sizeof(double) * kGpObs * nrep * 4L * ctx->num_sms);
  if (!ctx->gp_psi || !ctx->gp_psi1 || !ctx->gp_ht || !ctx->gp_ta || !ctx->gp_tb || !ctx->gp_v0 ||
      !ctx->gp_vm1 || !ctx->gp_v1 || !ctx->gp_vtot || !ctx->gp_ebar || !ctx->gp_active ||
      !ctx->gp_sact || !ctx->gp_coef || !ctx->gp_gram || !ctx->gp_obs ||
      (nocc <= kZgMaxN && !ctx->gp_zpart))
    return set_error(ctx, RMGTD_ENOMEM, "grid propagation buffers");
  if (ctx->nproj > 0) {
    const int rc = gp_f32(ctx) ? gp_build_kb_lists<float>(ctx) : gp_build_kb_lists<double>(ctx);
    if (rc) return rc;
  }
  ctx->gp_tma = gp_f32(ctx) ? gp_encode_term_maps<float>(ctx) : gp_encode_term_maps<double>(ctx);
  k_gp_init<<<gp_blocks(ctx, plane), 256, 0, ctx->stream>>>(ctx->phi, plane, nrep, ctx->gp_psi);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_init");
  // V_0 = V_-1 = V_H + V_xc of the starting density (computed by the set-up)
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_v0, ctx->vhxc, vsz, cudaMemcpyDeviceToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_vm1, ctx->vhxc, vsz, cudaMemcpyDeviceToDevice, ctx->stream));
  if (ctx->gp_vm2)   // V_-2 = V_0 too: the first steps' quadratic seed is the linear one
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_vm2, ctx->vhxc, vsz, cudaMemcpyDeviceToDevice, ctx->stream));
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

// fields of the orbitals `psi` for every replica: rho, V_H, V_xc, eps_xc, V_Hxc (ctx arrays);
// psi null (float32 terms): of the pass's psi_1 = psi0 + the series' sum, the density as a
// float32 change on rho0
static int gp_fields(rmgtd_ctx* ctx, const double* psi) {
  const long Ng = ctx->Ng;
  ph_begin(ctx, PH_RHO);
  if (psi) {
    k_gp_density<<<dim3(gp_blocks(ctx, Ng), ctx->nrep), 256, 0, ctx->stream>>>(psi, ctx->f_dev, ctx->N,
                                                                              Ng, ctx->rho);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_density");
  } else {
    k_gp_drho<<<dim3(gp_blocks(ctx, Ng), ctx->nrep), 256, 0, ctx->stream>>>(
        ctx->gp_psi0f, ctx->gp_acc, ctx->gp_f32occ, ctx->N, Ng, ctx->gp_rho0, ctx->rho);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_drho");
  }
  ph_end(ctx);
  int rc = RMGTD_OK;
  if (ctx->hartree_xc) {
    ph_begin(ctx, PH_HARTREE);
    rc = hartree_coop(ctx, ctx->rho, ctx->vh, nullptr, 0, ctx->nrep, 0);
    ph_end(ctx);
    if (rc) return rc;
  }
  ph_begin(ctx, PH_XC);
  rc = launch_lda(ctx, ctx->rho, ctx->hartree_xc ? ctx->vh : nullptr, 0, ctx->vxc, ctx->exc,
                  ctx->vhxc, nullptr, Ng, nullptr, ctx->nrep, Ng, ctx->hartree_xc);
  ph_end(ctx);
  return rc;
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
  double* out = ctx->gp_psi + 2 * r * plane;
  double* gre = ctx->gp_gram;
  double* gim = gre + NN;
  double* y = gim + NN;
  double* xre = y + NN;
  double* xim = xre + NN;
  // G_nm = h^3 sum psi_n conj(psi_m)
  if (N <= kZgMaxN) {
    const int nblk = gp_zgram_blocks(ctx);
    k_gp_zgram_partial<<<nblk, kZgThreads, 0, ctx->stream>>>(N, ctx->Ng, re, im, ctx->gp_zpart);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_zgram_partial");
    k_gp_zgram_reduce<<<gp_blocks(ctx, 32L * N * (N + 1) / 2), 256, 0, ctx->stream>>>(
        N, nblk, ctx->gp_zpart, ctx->h3, gre, gim);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_zgram_reduce");
  } else {   // Re = R R^T + I I^T, Im = Y - Y^T with Y = I R^T (the tiled float64 Gram)
    int rc = gram(ctx, re, re, nullptr, 0, 1, ctx->h3, nullptr, gre, nullptr, nullptr, 1, nullptr);
    if (!rc) rc = gram(ctx, im, im, nullptr, 0, 1, ctx->h3, gre, gre, nullptr, nullptr, 1, nullptr);
    if (!rc) rc = gram(ctx, im, re, nullptr, 0, 1, ctx->h3, nullptr, y, nullptr, nullptr, 0, nullptr);
    if (rc) return rc;
    k_gp_antisym<<<gp_blocks(ctx, NN), 256, 0, ctx->stream>>>(N, y, gim);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_antisym");
  }
  k_zcholesky<<<1, 1024, 0, ctx->stream>>>(N, gre, gim, ctx->status);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_zcholesky");
  if (N <= 32) {   // psi <- X psi1 with X = L^-1, the point's orbitals in registers
    k_ztri_inverse<<<1, 1024, 0, ctx->stream>>>(N, gre, gim, xre, xim);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_ztri_inverse");
    if (N <= 16)
      k_gp_xapply<16><<<gp_blocks(ctx, ctx->Ng), 256, 0, ctx->stream>>>(N, ctx->Ng, xre, xim, re, out);
    else
      k_gp_xapply<32><<<gp_blocks(ctx, ctx->Ng), 256, 0, ctx->stream>>>(N, ctx->Ng, xre, xim, re, out);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_xapply");
  } else {
    k_gp_fsubst<<<gp_blocks(ctx, ctx->Ng), 256, 0, ctx->stream>>>(N, ctx->Ng, gre, gim, re, out);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_fsubst");
  }
  return RMGTD_OK;
}

// the orbital series of every active replica for one pass: psi_1 = sum of the terms (tmax,
// tsum, status per replica)
template <typename T>
static int gp_series(rmgtd_ctx* ctx, const std::vector<int>& active, std::vector<int>& status,
                     std::vector<int>& tmax, std::vector<int>& tsum) {
  const int nrep = ctx->nrep;
  const long Ng = ctx->Ng, rplane = 2L * ctx->N * Ng;
  const double thr2 = ctx->opt.dP_thrs * ctx->opt.dP_thrs;
  k_gp_vtot<T><<<dim3(gp_blocks(ctx, Ng), nrep), 256, 0, ctx->stream>>>(
      ctx->vion, ctx->gp_v0, ctx->gp_v1, ctx->gp_ebar, (T*)ctx->gp_vtot, Ng, ctx->nx, ctx->ny,
      ctx->nz, ctx->h);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_vtot");
  T* ta = (T*)ctx->gp_ta;
  T* tb = (T*)ctx->gp_tb;
  const T* tin = ta;   // the term's input and output (the first from psi)
  T* tout = tb;
  if constexpr (sizeof(T) == sizeof(float)) {   // the step's psi in float32, converted once
    tin = ctx->gp_psi0f;
    tout = ta;
  } else {
    k_gp_start<T><<<dim3(gp_blocks(ctx, rplane), nrep), 256, 0, ctx->stream>>>(
        ctx->gp_psi, ctx->gp_psi1, ta, rplane, ctx->gp_active);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_start");
  }
  // the terms in batches between read-backs of the device-side stopping test: the first
  // batch as long as the last series less one, then two at a time (terms queued after a
  // series has stopped return at once)
  std::vector<int> ctl(3 * nrep, 0);
  for (int r = 0; r < nrep; ++r) ctl[r] = active[r];
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_sact, ctl.data(), sizeof(int) * 3 * nrep,
                                  cudaMemcpyHostToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->errbits, 0, sizeof(unsigned long long) * nrep, ctx->stream));
  int batch = std::max(1, ctx->gp_terms_hint - 1);
  for (int k = 1;;) {
    for (int b = 0; b < batch; ++b, ++k) {
      int rc = gp_term<T>(ctx, tin, tout, ctx->opt.dt / k, k == 1);
      if (rc) return rc;
      tin = tout;
      tout = tout == ta ? tb : ta;
      k_gp_series_ctl<<<1, 32, 0, ctx->stream>>>(nrep, k, thr2, ctx->opt.max_terms, ctx->gp_sact,
                                                 ctx->errbits);
      ++ctx->launches;
      RMGTD_LAUNCH(ctx, "k_gp_series_ctl");
    }
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctl.data(), ctx->gp_sact, sizeof(int) * 3 * nrep,
                                    cudaMemcpyDeviceToHost, ctx->stream));
    RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    bool more = false;
    for (int r = 0; r < nrep; ++r) more = more || ctl[r];
    if (!more) break;
    batch = 2;
  }
  int last = 0;
  for (int r = 0; r < nrep; ++r) {
    if (!active[r]) continue;
    const int terms = ctl[2 * nrep + r];
    if (ctl[nrep + r]) status[r] = ctl[nrep + r];
    tmax[r] = std::max(tmax[r], terms);
    tsum[r] += terms;
    last = std::max(last, terms);
  }
  ctx->gp_terms_hint = last;
  return RMGTD_OK;
}

int gridprop_step(rmgtd_ctx* ctx, rmgtd_stats* st) {
  const int nrep = ctx->nrep;
  const long Ng = ctx->Ng;
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
  k_gp_extrap<<<vb, 256, 0, ctx->stream>>>(ctx->gp_v0, ctx->gp_vm1, ctx->gp_vm2, ctx->gp_v1, Ng * nrep);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gp_extrap");
  const bool f32 = gp_f32(ctx);
  const long rplane = 2L * ctx->N * Ng;
  if (ctx->hartree_xc) {   // the first solve's guess: V_H extrapolated one step ahead
    k_gp_vh_guess<<<vb, 256, 0, ctx->stream>>>(ctx->vh, ctx->gp_vh1, ctx->gp_vh2, ctx->gp_vh_hist,
                                               Ng * nrep);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_vh_guess");
    ctx->gp_vh_hist = std::min(2, ctx->gp_vh_hist + 1);
  }
  if (f32) {   // the step's psi in float32 and its density in float64, once per step
    k_gp_to_f32<<<gp_blocks(ctx, rplane * nrep), 256, 0, ctx->stream>>>(ctx->gp_psi, ctx->gp_psi0f,
                                                                         rplane * nrep);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_to_f32");
    k_gp_density<<<dim3(gp_blocks(ctx, Ng), nrep), 256, 0, ctx->stream>>>(ctx->gp_psi, ctx->f_dev, ctx->N,
                                                                         Ng, ctx->gp_rho0);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_density");
  }
  std::vector<int> active(nrep, 1), passes(nrep, 0), tmax(nrep, 0), tsum(nrep, 0), status(nrep, 0);
  std::vector<double> herr(nrep, 0.0), m;
  bool any = true;
  for (int pass = 1; pass <= ctx->opt.max_scf && any; ++pass) {
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->gp_active, active.data(), sizeof(int) * nrep,
                                    cudaMemcpyHostToDevice, ctx->stream));
    ph_begin(ctx, PH_ELDYN);   // the orbital series takes the commutator series' place
    int rc = f32 ? gp_series<float>(ctx, active, status, tmax, tsum)
                 : gp_series<double>(ctx, active, status, tmax, tsum);
    ph_end(ctx);
    if (rc) return rc;
    for (int r = 0; r < nrep; ++r)
      if (status[r]) active[r] = 0;
    // V_new of the propagated orbitals; H_err = max|V_new - V_1|
    rc = gp_fields(ctx, f32 ? nullptr : ctx->gp_psi1);
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
  ph_begin(ctx, PH_OTHER);
  if (f32) {   // psi_1 = psi + hi + lo of every replica's last series
    k_gp_fold<<<dim3(gp_blocks(ctx, rplane), nrep), 256, 0, ctx->stream>>>(
        ctx->gp_psi, ctx->gp_acc, rplane * nrep, ctx->gp_psi1, rplane, nullptr);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_gp_fold");
  }
  for (int r = 0; r < nrep; ++r) {
    int rc = gp_orthonormalize(ctx, r);
    if (rc) return rc;
  }
  ph_end(ctx);
  int cst = 0;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(&cst, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  // V_-1 <- V_0, V_0 <- V_1 (rotate the buffers)
  if (ctx->gp_vm2) std::swap(ctx->gp_vm2, ctx->gp_vm1);   // V_-2 <- V_-1
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
