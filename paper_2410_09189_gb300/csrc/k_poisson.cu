// Hartree potential: Lap_12 V_H = -4 pi rho on the grid (Section 2.1; Algorithm 1's density-functional update).
//
// Discrete problem (the same one the kinetic stencil defines): interior unknowns, ghost
// layers holding the monopole + dipole field of rho about the box centre,
//   (-Lap_12^0) V = 4 pi rho + L_ghost(V_b),  V_b(r) = Q/|r| + p.r/|r|^3.
// The ghost term is linear in (Q, p): L_ghost(V_b) = Q G0 + px Gx + py Gy + pz Gz with four
// grid fields G fixed by the grid, formed once at set-up.
//
// Solver: flexible (Polak-Ribiere) conjugate gradients.  Default preconditioner: the 3-D
// sine transform (DST-I) that diagonalises the Toeplitz part of the 12th-order operator,
// applied in float32 as five passes of 1-D transforms on the tensor cores (TF32 MMAs); the
// operator with zero ghosts differs from that part only next to the faces, so CG needs a
// few iterations (1.6-1.7 per solve on the 64^3 ring against 2.9 with the V-cycle).  Where
// its tables do not fit in shared memory, or on request, one multigrid V-cycle in float32
// (the paper's multigrid, Section 2.1): cell-centred coarsening by 2 down to <= 64 points,
// 7-point operators at spacing 2^l h, damped Jacobi smoothing (2 pre, 2 post), trilinear
// prolongation and the box restriction (mean over the 8 children, formed in the same pass
// as the residual; the V-cycle is then not symmetric, which flexible CG tolerates); the
// levels with <= 4096 points run inside single blocks, whose coarsest level is solved
// exactly.  The float64 path iterates
// on V itself; the mixed path iterates in float32 on the change of V relative to the
// reference potential, with float32 right-hand side and dot products summed per warp in
// float32 and across warps and blocks in float64 (float64 runs at a small fraction of the
// float32 rate on this GPU, so no per-point float64 work remains in that solve).
//
// One cooperative launch runs the whole solve: prologue, every CG iteration and every
// preconditioner phase, separated by grid barriers (7 per iteration with the sine
// transform, 11 with the V-cycle at 64^3).  A p = A z +
// beta A p_old is carried as a vector, so the 37-point operator is applied once per
// iteration to z, and (p, A p) follows from four dot products taken with A z.  Every block
// sums the per-block partials of a reduction in the same order, so all blocks take the
// same decisions and the result does not depend on timing.  Float32 level-0 passes work on
// quads (4 consecutive x-points per thread, 16-byte loads).  In the mixed pass the prologue
// takes the multipole moments of the density change from the density kernel, and a closing
// phase forms the pass's potential change dV_H + dV_xc (the float32 xc increment).
#include <math.h>

#include "fastdiv.h"
#include "lda.cuh"
#include "rmgtd_internal.cuh"

namespace rmgtd {

constexpr double kPi = 3.14159265358979323846;
constexpr float kJacobiW = 6.0f / 7.0f;
constexpr int kTailMax = 4096;
constexpr size_t kDstSmemMax = 160 * 1024;   // sine-transform preconditioner: larger grids
                                              // fall back to the multigrid V-cycle
constexpr int kCoarseDirect = 64;   // a level below the finest with at most this many points is
                                    // the coarsest (solved exactly with its precomputed inverse)
// The sine-transform preconditioner's folded matrices for lines of n points, as tensor-core
// A operands: kn x kn (kn = ceil(n/2) for the even outputs, floor(n/2) for the odd ones),
// output-major with rows padded to 16 and a row stride of 4 mod 32 words covering kn rounded
// up to 8 (zero padding), so the m16n8k8 fragment loads hit 32 distinct banks.
__host__ __device__ inline int dst_astride(int kn) { return 32 * ((((kn + 7) & ~7) + 27) / 32) + 4; }
__host__ __device__ inline int dst_arows(int kn) { return (kn + 15) & ~15; }
__host__ __device__ inline int dst_mat_floats(int n) {
  const int hp = (n + 1) >> 1, h = n >> 1;
  return dst_arows(hp) * dst_astride(hp) + dst_arows(h) * dst_astride(h);
}
// tile columns for W lines: W rounded up to 8, and to 8 or 24 mod 32 (conflict-free B loads)
__host__ __device__ inline int dst_wpad(int W) {
  int Wp = (W + 7) & ~7;
  if ((Wp & 31) == 0 || (Wp & 31) == 16) Wp += 8;
  return Wp;
}
constexpr int kPre = 2, kPost = 2, kCoarseSweeps = 40;
static_assert(kPre == 2, "the pre-smoothing pass fuses exactly two sweeps from zero");
// relative residual of the float32 correction solve of the mixed path: the unknown is the
// change of V_H relative to the reference potential (|dV_H| ~ 1e-3 after a 1e-3 kick), so
// 3e-6 of it is ~3e-9 absolute -- far below the SCF threshold H_thrs that decides the step
constexpr double kMixedPoissonTol = 3e-6;

struct Grid3 {
  int nx, ny, nz;
  double h;
};

constexpr int kMaxLevels = 12;
// one multi-block level of the hierarchy, replicas stacked: [rep][n]
struct Level {
  int nx, ny, nz, n;
  float h2;
  FastDiv dx, dy, dn;     // division by nx, ny, n
  float *x, *b, *t;
};
// levels solved inside one block (no replica stride: one block per replica)
struct Tail {
  int nl;
  int nx[kMaxLevels], ny[kMaxLevels], nz[kMaxLevels], n[kMaxLevels];
  float h2[kMaxLevels];
  FastDiv dx[kMaxLevels], dy[kMaxLevels];
};
struct LevelTable {
  int nl;       // all levels
  int nmulti;   // levels [0, nmulti) run across the grid; [nmulti, nl) inside one block
  Level L[kMaxLevels];
  Tail T;
};

__device__ __forceinline__ void xyz_of(int g, int nx, int ny, const FastDiv& dx,
                                       const FastDiv& dy, int& ix, int& iy, int& iz) {
  const int q = fdiv(g, dx);
  ix = g - q * nx;
  iz = fdiv(q, dy);
  iy = q - iz * ny;
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

// ---- the 12th-order operator A = -Lap_12 with zero ghosts -------------------------------
template <typename V>
__device__ __forceinline__ V apply_A12(const V* __restrict__ x, int ix, int iy, int iz, int nx,
                                       int ny, int nz, V ih2) {
  const int plane = nx * ny;
  const int g = iz * plane + iy * nx + ix;
  V s = (V)(3.0 * fd_coef(0)) * x[g];
#pragma unroll
  for (int m = 1; m <= kFdRadius; ++m) {
    V t = 0;
    if (ix + m < nx) t += x[g + m];
    if (ix - m >= 0) t += x[g - m];
    if (iy + m < ny) t += x[g + m * nx];
    if (iy - m >= 0) t += x[g - m * nx];
    if (iz + m < nz) t += x[g + m * plane];
    if (iz - m >= 0) t += x[g - m * plane];
    s = fma((V)fd_coef(m), t, s);
  }
  return -s * ih2;
}

// ---- multigrid in float32 (7-point operators, zero Dirichlet ghosts) ----------------------
__device__ __forceinline__ float lap7f(const float* __restrict__ x, int ix, int iy, int iz,
                                       int nx, int ny, int nz, float* center) {
  const int plane = nx * ny;
  const int g = iz * plane + iy * nx + ix;
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

// ---- quads: 4 consecutive x-points per thread (float32, nx a multiple of 4) -----------------
// A thread loads whole 16-byte vectors of its row and of the neighbouring rows instead of
// scalar neighbours, so one quad of a stencil needs 7 (7-point) or 29 (37-point) vector loads
// instead of 28 or 148 scalar ones, with all of them in flight together.  Sums keep the
// scalar kernels' order (+x, -x, +y, -y, +z, -z; absent neighbours add zero).
__device__ __forceinline__ uint32_t saddr_f(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ float4 ld4_if(bool c, const float* p) {
  return c ? ld4(p) : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ float f4(const float4& v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// h^2 (-Lap_7 x) of the quad starting at g0 (x = ix0 .. ix0 + 3); c4 receives x there
__device__ __forceinline__ float4 lap7_quad(const float* __restrict__ x, int g0, int ix0, int iy,
                                            int iz, int nx, int ny, int nz, float4& c4) {
  const int plane = nx * ny;
  c4 = ld4(x + g0);
  const float xl = ix0 > 0 ? x[g0 - 1] : 0.0f;
  const float xr = ix0 + 4 < nx ? x[g0 + 4] : 0.0f;
  const float4 yp = ld4_if(iy + 1 < ny, x + g0 + nx), ym = ld4_if(iy > 0, x + g0 - nx);
  const float4 zp = ld4_if(iz + 1 < nz, x + g0 + plane), zm = ld4_if(iz > 0, x + g0 - plane);
  float4 r;
  r.x = 6.0f * c4.x - (((((c4.y + xl) + yp.x) + ym.x) + zp.x) + zm.x);
  r.y = 6.0f * c4.y - (((((c4.z + c4.x) + yp.y) + ym.y) + zp.y) + zm.y);
  r.z = 6.0f * c4.z - (((((c4.w + c4.y) + yp.z) + ym.z) + zp.z) + zm.z);
  r.w = 6.0f * c4.w - (((((xr + c4.z) + yp.w) + ym.w) + zp.w) + zm.w);
  return r;
}

// A12 x (the 37-point operator of apply_A12) on the quad; c4 receives x there
__device__ __forceinline__ float4 A12_quad(const float* __restrict__ x, int g0, int ix0, int iy,
                                           int iz, int nx, int ny, int nz, float ih2, float4& c4) {
  const int plane = nx * ny;
  float xl[20];   // x - 8 .. x + 11 of the row, zero outside it
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int xo = ix0 - 8 + 4 * k;
    const float4 v = ld4_if(xo >= 0 && xo < nx, x + g0 - 8 + 4 * k);
    xl[4 * k] = v.x;
    xl[4 * k + 1] = v.y;
    xl[4 * k + 2] = v.z;
    xl[4 * k + 3] = v.w;
  }
  c4 = make_float4(xl[8], xl[9], xl[10], xl[11]);
  const float c0 = (float)(3.0 * fd_coef(0));
  float sm[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) sm[q] = c0 * xl[8 + q];
#pragma unroll
  for (int m = 1; m <= kFdRadius; ++m) {
    const float4 yp = ld4_if(iy + m < ny, x + g0 + m * nx);
    const float4 ym = ld4_if(iy - m >= 0, x + g0 - m * nx);
    const float4 zp = ld4_if(iz + m < nz, x + g0 + m * plane);
    const float4 zm = ld4_if(iz - m >= 0, x + g0 - m * plane);
    const float cm = (float)fd_coef(m);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float t = ((((xl[8 + q + m] + xl[8 + q - m]) + f4(yp, q)) + f4(ym, q)) + f4(zp, q)) +
                      f4(zm, q);
      sm[q] = fmaf(cm, t, sm[q]);
    }
  }
  return make_float4(-sm[0] * ih2, -sm[1] * ih2, -sm[2] * ih2, -sm[3] * ih2);
}

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

// Box restriction of the residual: the mean of b - A x over the 8 fine children of coarse
// point (I, J, K) (cell-centred coarsening by 2; A = 7-point operator / h^2).
__device__ __forceinline__ float restrict_residual(const float* __restrict__ x,
                                                   const float* __restrict__ b, int I, int J,
                                                   int K, int nx, int ny, int nz, float ih2) {
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int fx = 2 * I + (c & 1), fy = 2 * J + ((c >> 1) & 1), fz = 2 * K + (c >> 2);
    float cc;
    const float ax = lap7f(x, fx, fy, fz, nx, ny, nz, &cc) * ih2;
    s += b[(fz * ny + fy) * nx + fx] - ax;
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
  auto at = [&](int i, int j, int k) { return xc[(k * cy + j) * cx + i]; };
  return wz0 * (wy0 * (wx0 * at(x0, y0, z0) + wx1 * at(x1, y0, z0)) +
                wy1 * (wx0 * at(x0, y1, z0) + wx1 * at(x1, y1, z0))) +
         wz1 * (wy0 * (wx0 * at(x0, y0, z1) + wx1 * at(x1, y0, z1)) +
                wy1 * (wx0 * at(x0, y1, z1) + wx1 * at(x1, y1, z1)));
}

// Trilinear prolongation of the coarse correction onto the fine quad x0 .. x0 + 3 (x0 a
// multiple of 4) of row (fy, fz): the quad reads coarse x I0 - 1 .. I0 + 2 (I0 = x0 / 2) of
// its 2 x 2 coarse lines once; weights and sums as prolong_point.
__device__ __forceinline__ float4 prolong_quad(const float* __restrict__ xc, int x0, int fy,
                                               int fz, int cx, int cy, int cz) {
  const int I0 = x0 >> 1;
  int y0, y1, z0, z1;
  float wy0, wy1, wz0, wz1;
  tri_w(fy, cy, &y0, &y1, &wy0, &wy1);
  tri_w(fz, cz, &z0, &z1, &wz0, &wz1);
  const bool lok = I0 > 0, rok = I0 + 2 < cx;
  const float wl = lok ? 0.25f : 0.0f, wr = rok ? 0.25f : 0.0f;
  float h[4][4];   // [line][fine q]: x-interpolated coarse line (y0 z0, y1 z0, y0 z1, y1 z1)
#pragma unroll
  for (int ln = 0; ln < 4; ++ln) {
    const int j = (ln & 1) ? y1 : y0, k = (ln & 2) ? z1 : z0;
    const float* row = xc + (k * cy + j) * cx;
    const float v0 = row[I0], v1 = row[I0 + 1];
    const float vl = row[lok ? I0 - 1 : I0], vr = row[rok ? I0 + 2 : I0 + 1];
    h[ln][0] = 0.75f * v0 + wl * vl;
    h[ln][1] = 0.75f * v0 + 0.25f * v1;
    h[ln][2] = 0.75f * v1 + 0.25f * v0;
    h[ln][3] = 0.75f * v1 + wr * vr;
  }
  float r[4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
    r[q] = wz0 * (wy0 * h[0][q] + wy1 * h[1][q]) + wz1 * (wy0 * h[2][q] + wy1 * h[3][q]);
  return make_float4(r[0], r[1], r[2], r[3]);
}

// ---- coarse tail of the V-cycle inside one block (levels with <= kTailMax points) ---------
__device__ void tail_jacobi(const Tail& L, int l, float* x, float* t, const float* b,
                            int first) {
  const int nx = L.nx[l], ny = L.ny[l], nz = L.nz[l], n = L.n[l];
  const float h2 = L.h2[l], c = kJacobiW * h2 / 6.0f, ih2 = 1.0f / h2;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    if (first) {
      t[g] = c * b[g];
    } else {
      int ix, iy, iz;
      xyz_of(g, nx, ny, L.dx[l], L.dy[l], ix, iy, iz);
      float cc;
      const float ax = lap7f(x, ix, iy, iz, nx, ny, nz, &cc) * ih2;
      t[g] = cc + c * (b[g] - ax);
    }
  }
  __syncthreads();
  for (int g = threadIdx.x; g < n; g += blockDim.x) x[g] = t[g];
  __syncthreads();
}

// V-cycle of the tail levels for one replica inside one block (all threads of the block):
// b_in / x_out are that replica's arrays of the first tail level (x_out NULL: the result
// stays in shared memory, at sm), sm the dynamic shared memory, cinv the transposed inverse
// of the coarsest level's operator in shared memory (NULL: Jacobi sweeps there).  Down: both pre-sweeps from zero in one pass, residual, restriction; up:
// prolongation, two post-sweeps ping-ponging between x and t.
__device__ void tail_vcycle(const Tail& L, const float* __restrict__ b_in,
                            float* __restrict__ x_out, const float* __restrict__ cinv, float* sm) {
  float* xs[kMaxLevels];
  float* bs[kMaxLevels];
  float* ts[kMaxLevels];
  int off = 0;
  for (int l = 0; l < L.nl; ++l) {
    xs[l] = sm + off;
    bs[l] = sm + off + L.n[l];
    ts[l] = sm + off + 2 * L.n[l];
    off += 3 * L.n[l];
  }
  const int n0 = L.n[0];
  for (int g = threadIdx.x; g < n0; g += blockDim.x) bs[0][g] = b_in[g];
  __syncthreads();
  for (int l = 0; l < L.nl; ++l) {
    const bool coarsest = (l == L.nl - 1);
    if (coarsest && cinv) {
      // exact solve with the precomputed inverse of the coarsest operator (cinv: its
      // transpose in shared memory, so a warp reads 32 consecutive words per j)
      const int nc = L.n[l];
      for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        float a = 0.0f;
        for (int j = 0; j < nc; ++j) a = fmaf(cinv[j * nc + i], bs[l][j], a);
        xs[l][i] = a;
      }
      __syncthreads();
      break;
    }
    if (coarsest) {
      for (int sw = 0; sw < kCoarseSweeps; ++sw) tail_jacobi(L, l, xs[l], ts[l], bs[l], sw == 0);
      break;
    }
    const int nx = L.nx[l], ny = L.ny[l], nz = L.nz[l], n = L.n[l];
    const float h2 = L.h2[l], ih2 = 1.0f / h2, c = kJacobiW * h2 / 6.0f;
    if ((nx & 3) == 0) {   // quads (the level's arrays start at multiples of 4 floats)
      for (int g0 = 4 * threadIdx.x; g0 < n; g0 += 4 * blockDim.x) {
        int ix, iy, iz;
        xyz_of(g0, nx, ny, L.dx[l], L.dy[l], ix, iy, iz);
        float4 bc;
        const float4 ab = lap7_quad(bs[l], g0, ix, iy, iz, nx, ny, nz, bc);
        *reinterpret_cast<float4*>(xs[l] + g0) = make_float4(
            c * (2.0f * bc.x - c * (ab.x * ih2)), c * (2.0f * bc.y - c * (ab.y * ih2)),
            c * (2.0f * bc.z - c * (ab.z * ih2)), c * (2.0f * bc.w - c * (ab.w * ih2)));
      }
    } else {
      for (int g = threadIdx.x; g < n; g += blockDim.x) {   // x = c (2 b - c A b)
        int ix, iy, iz;
        xyz_of(g, nx, ny, L.dx[l], L.dy[l], ix, iy, iz);
        float bc;
        const float ab = lap7f(bs[l], ix, iy, iz, nx, ny, nz, &bc) * ih2;
        xs[l][g] = c * (2.0f * bc - c * ab);
      }
    }
    __syncthreads();
    const int cx = L.nx[l + 1], cy = L.ny[l + 1], nc = L.n[l + 1];
    for (int g = threadIdx.x; g < nc; g += blockDim.x) {   // restricted residual
      int I, J, K;
      xyz_of(g, cx, cy, L.dx[l + 1], L.dy[l + 1], I, J, K);
      bs[l + 1][g] = restrict_residual(xs[l], bs[l], I, J, K, nx, ny, nz, ih2);
    }
    __syncthreads();
  }
  for (int l = L.nl - 2; l >= 0; --l) {
    const int nx = L.nx[l], ny = L.ny[l], nz = L.nz[l], n = L.n[l];
    const int cx = L.nx[l + 1], cy = L.ny[l + 1], cz = L.nz[l + 1];
    const float h2 = L.h2[l], ih2 = 1.0f / h2, c = kJacobiW * h2 / 6.0f;
    const bool quad = (nx & 3) == 0;
    if (quad) {
      for (int g0 = 4 * threadIdx.x; g0 < n; g0 += 4 * blockDim.x) {
        int fx, fy, fz;
        xyz_of(g0, nx, ny, L.dx[l], L.dy[l], fx, fy, fz);
        const float4 pq = prolong_quad(xs[l + 1], fx, fy, fz, cx, cy, cz);
        float4 v = ld4(xs[l] + g0);
        v.x += pq.x;
        v.y += pq.y;
        v.z += pq.z;
        v.w += pq.w;
        *reinterpret_cast<float4*>(xs[l] + g0) = v;
      }
    } else {
      for (int g = threadIdx.x; g < n; g += blockDim.x) {
        int fx, fy, fz;
        xyz_of(g, nx, ny, L.dx[l], L.dy[l], fx, fy, fz);
        xs[l][g] += prolong_point(xs[l + 1], fx, fy, fz, cx, cy, cz);
      }
    }
    __syncthreads();
    for (int sw = 0; sw < kPost; ++sw) {
      const float* in = (sw & 1) ? ts[l] : xs[l];
      float* out = (sw & 1) ? xs[l] : ts[l];
      if (quad) {
        for (int g0 = 4 * threadIdx.x; g0 < n; g0 += 4 * blockDim.x) {
          int ix, iy, iz;
          xyz_of(g0, nx, ny, L.dx[l], L.dy[l], ix, iy, iz);
          float4 cc;
          const float4 ax = lap7_quad(in, g0, ix, iy, iz, nx, ny, nz, cc);
          const float4 bv = ld4(bs[l] + g0);
          *reinterpret_cast<float4*>(out + g0) = make_float4(
              cc.x + c * (bv.x - ax.x * ih2), cc.y + c * (bv.y - ax.y * ih2),
              cc.z + c * (bv.z - ax.z * ih2), cc.w + c * (bv.w - ax.w * ih2));
        }
      } else {
        for (int g = threadIdx.x; g < n; g += blockDim.x) {
          int ix, iy, iz;
          xyz_of(g, nx, ny, L.dx[l], L.dy[l], ix, iy, iz);
          float cc;
          const float ax = lap7f(in, ix, iy, iz, nx, ny, nz, &cc) * ih2;
          out[g] = cc + c * (bs[l][g] - ax);
        }
      }
      __syncthreads();
    }
    if (kPost & 1)
      for (int g = threadIdx.x; g < n; g += blockDim.x) xs[l][g] = ts[l][g];
    __syncthreads();
  }
  if (x_out)
    for (int g = threadIdx.x; g < n0; g += blockDim.x) x_out[g] = xs[0][g];
  __syncthreads();
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
  // transposed: out[j n + i] = Minv[i][j] (the tail's threads i read consecutive words)
  for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x)
    out[(e % n) * n + e / n] = (float)Minv[e];
}

// ---- host set-up ---------------------------------------------------------------------------
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
    if ((int)ctx->mg.size() >= kMaxLevels) break;
    if ((nx & 1) || (ny & 1) || (nz & 1) || nx < 4 || ny < 4 || nz < 4) break;
    if (ctx->mg.size() >= 2 && L.n <= kCoarseDirect) break;
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
  // the coarsest level's inverse joins them when it is small (read from global otherwise)
  ctx->mg_cinv_smem = 0;
  if (ctx->mg_tail_level >= 0 && ctx->mg[nl - 1].n <= kCoarseDirect) {
    smem += sizeof(float) * ctx->mg[nl - 1].n * ctx->mg[nl - 1].n;
    ctx->mg_cinv_smem = 1;
  }
  ctx->mg_tail_smem = smem;
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
  // level table of the persistent solve (device copy, read once per launch)
  LevelTable lt;
  memset(&lt, 0, sizeof(lt));
  lt.nl = nl;
  lt.nmulti = ctx->mg_tail_level >= 0 ? ctx->mg_tail_level : nl;
  for (int l = 0; l < nl; ++l) {
    const MgLevel& M = ctx->mg[l];
    Level& L = lt.L[l];
    L.nx = M.nx;
    L.ny = M.ny;
    L.nz = M.nz;
    L.n = (int)M.n;
    L.h2 = (float)(M.h * M.h);
    L.dx = make_fastdiv(M.nx);
    L.dy = make_fastdiv(M.ny);
    L.dn = make_fastdiv((int)M.n);
    L.x = M.x;
    L.b = M.b;
    L.t = M.t;
  }
  if (ctx->mg_tail_level >= 0) {
    lt.T.nl = nl - lt.nmulti;
    for (int l = lt.nmulti; l < nl; ++l) {
      const MgLevel& M = ctx->mg[l];
      const int k = l - lt.nmulti;
      lt.T.nx[k] = M.nx;
      lt.T.ny[k] = M.ny;
      lt.T.nz[k] = M.nz;
      lt.T.n[k] = (int)M.n;
      lt.T.h2[k] = (float)(M.h * M.h);
      lt.T.dx[k] = make_fastdiv(M.nx);
      lt.T.dy[k] = make_fastdiv(M.ny);
    }
  }
  ctx->mg_table = dev_alloc(ctx, sizeof(LevelTable));
  if (!ctx->mg_table) return set_error(ctx, RMGTD_ENOMEM, "level table");
  RMGTD_CUDA(ctx, cudaMemcpy(ctx->mg_table, &lt, sizeof(LevelTable), cudaMemcpyHostToDevice));

  // sine-transform preconditioner tables: S_x, S_y, S_z (float32, row stride n rounded up to
  // 4, zero padding) and the 1-D eigenvalues lx, ly, lz of the 12th-order operator's Toeplitz
  // part, l[k] = -(a_0 + 2 sum_m a_m cos(m theta_k)) / h^2, theta_k = pi (k+1) / (n+1)
  {
    const int dims[3] = {ctx->nx, ctx->ny, ctx->nz};
    size_t nS = 0;
    for (int ax = 0; ax < 3; ++ax) nS += (size_t)dst_mat_floats(dims[ax]);
    std::vector<float> tab(nS + dims[0] + dims[1] + dims[2], 0.0f);
    size_t o = 0, ol = nS;
    for (int ax = 0; ax < 3; ++ax) {
      const int n = dims[ax], hp = (n + 1) / 2, h = n / 2;
      const int ase = dst_astride(hp), aso = dst_astride(h);
      // S[j][k] rounded to TF32 (nearest, ties to even: 10 explicit mantissa bits)
      auto S = [&](int j, int k) {
        const float v = (float)std::sin(kPi * (double)(j + 1) * (k + 1) / (n + 1));
        uint32_t u;
        memcpy(&u, &v, 4);
        u += 0xFFFu + ((u >> 13) & 1u);
        u &= 0xFFFFE000u;
        float r;
        memcpy(&r, &u, 4);
        return r;
      };
      for (int i = 0; i < hp; ++i)
        for (int k = 0; k < hp; ++k) tab[o + (size_t)i * ase + k] = S(2 * i, k);
      const size_t oo = o + (size_t)dst_arows(hp) * ase;
      for (int i = 0; i < h; ++i)
        for (int k = 0; k < h; ++k) tab[oo + (size_t)i * aso + k] = S(2 * i + 1, k);
      for (int k = 0; k < n; ++k) {
        const double th = kPi * (k + 1) / (n + 1);
        double sym = fd_coef(0);
        for (int m = 1; m <= kFdRadius; ++m) sym += 2.0 * fd_coef(m) * std::cos(m * th);
        tab[ol + k] = (float)(-sym / (ctx->h * ctx->h));
      }
      o += (size_t)dst_mat_floats(n);
      ol += n;
    }
    ctx->dst_tab = (float*)dev_alloc(ctx, sizeof(float) * tab.size());
    if (!ctx->dst_tab) return set_error(ctx, RMGTD_ENOMEM, "sine-transform tables");
    RMGTD_CUDA(ctx, cudaMemcpy(ctx->dst_tab, tab.data(), sizeof(float) * tab.size(),
                               cudaMemcpyHostToDevice));
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

// slot capacity of the reduction partials (grid-stride kernels and the persistent solve)
int poisson_red_cap(int num_sms, int red_blocks) { return std::max(num_sms, red_blocks); }

// ---- the persistent solve ---------------------------------------------------------------
namespace coop {

constexpr int kThreadsC = 1024;
constexpr int kWarps = kThreadsC / 32;
constexpr int kMaxRep = 32;
constexpr int kMaxDots = 4;     // dot products reduced together in one phase
constexpr int kSlots = 8;
// reduction slots per replica: 0 (b,b)  1 (r,r)  2 (r,z)  3 (z,Az)  4 (z,Ap_old) / Q
// 5 (p_old,Az) / px  6 (r_new,z_old) / py  7 pz   (moments only in the prologue)

template <typename V>
struct Args {
  const LevelTable* lt;   // device copy of the level table
  int nrep;
  double h;
  const double* rho;      // float64 path: density [rep][n0]
  const float* drho;      // mixed path: density change rho - rho_ref [rep][n0]
  const double* gf;       // float64 ghost response fields [4][n0]
  const float* gf32;      // float32 copy (mixed path)
  const float* cinv;
  int cinv_smem;          // copy cinv next to the tail levels in shared memory
  // sine-transform preconditioner instead of the V-cycle (dst != 0): S_x, S_y, S_z (row
  // strides rounded up to 4) then lx, ly, lz, in global memory; copied to shared memory
  int dst;
  int dst_wb;             // lines per batch of a transform pass
  const float* dst_tab;
  int zero_bc;
  V* x;                   // unknown (initial guess in, solution out) [rep][n0]
  V *r, *z, *p, *Ap, *Az;
  double* part;           // [rep][kSlots][gridDim.x] per-block partial sums
  PcgState* st;
  const RepCtl* ctl;
  double tol;
  int max_it;
  unsigned* bar;
  int* status;
  unsigned long long* counters;   // [0] solves, [1] CG iterations (summed over replicas)
  int vec4;               // float path with nx % 4 == 0: level-0 phases on quads
  // float path: closing phase dv_out = x + V_xc(rho0 + drho) - V_xc(rho0) (the mixed pass's
  // potential change; rho0f = rho0 rounded to float32), when dv_out is set
  const double* rho0;
  const float* rho0f;
  float* dv_out;
  // moments of the density change already formed by the density kernel: [rep][4][nmom]
  // per-CTA partials (NULL: the prologue forms them)
  const double* mom;
  int nmom;
};

// ---- sine-transform preconditioner (float32) ------------------------------------------------
// z = M r with M = S (Lambda^-1 (S r)) scaled by 8 / ((nx+1)(ny+1)(nz+1)): S is the 3-D DST-I
// (per axis S_n[j][k] = sin(pi (j+1)(k+1) / (n+1)), symmetric, S_n S_n = (n+1)/2 I) and
// Lambda(kx, ky, kz) = lx[kx] + ly[ky] + lz[kz] the eigenvalues of the Toeplitz part of the
// 12th-order operator, l[k] = -(a_0 + 2 sum_m a_m cos(m theta_k)) / h^2, theta_k =
// pi (k+1) / (n+1).  The operator with zero ghosts differs from that Toeplitz part only in the
// rows within the stencil radius of a face, so M A has its spectrum close to 1 (the CG
// residual falls by ~0.03-0.07 per iteration, against ~0.25 with the 7-point V-cycle).
// One application is five passes of 1-D transforms (x, y, z with the scaling and the inverse
// z, y, x), each over every line of the grid along its axis, split evenly over the blocks.
// The matrices are stored folded: S[j][n-1-k] = (-1)^j S[j][k], so with the line's sums
// P_k = x_k + x_{n-1-k} (k < n/2; P of the middle point of an odd line is that point) and
// differences M_k = x_k - x_{n-1-k} (both formed while the MMA operands are loaded), the even
// outputs are Se P and the odd ones So M, with
// Se[i][k] = S[2i][k] (ceil(n/2) x ceil(n/2)) and So[i][k] = S[2i+1][k] (floor(n/2) squared):
// half the multiply-adds and half the table of a plain product.  The products run on the
// tensor cores as warp-level m16n8k8 TF32 MMAs (float32 accumulation; the tables are stored
// already rounded to TF32): they are 16 x 88 x 32 tiles inside the persistent solve, where a
// warp's MMA and its fragment loads cost less than any staging for larger tiles would.
// (dst_astride, dst_arows, dst_mat_floats and dst_wpad, the tables' and tiles' layout, are
// defined at the top of this file)

// One pass along axis ax over this block's share of the lines (all threads of the block),
// in batches of at most wb lines: out(line, j) = sum_k S[j][k] in(line, k); with scale
// (z axis): forward, times norm / Lambda, inverse.  S: this axis's folded matrices Se, So in
// shared memory; tA, tB: shared tiles of n x Wp floats (Wp = dst_wpad(the batch's line
// count)); lbase, lxy: shared scratch of one int / float per line of a batch.  Flat indices are split into (row,
// column) incrementally (no division per element); int offsets (nrep n0 < 2^31).
template <typename VI, typename VO>
__device__ void dst_pass(int ax, const VI* __restrict__ in, VO* __restrict__ out, int nrep,
                         int nx, int ny, int nz, const float* S, float* tA, float* tB,
                         int* lbase, float* lxy, bool scale, const float* __restrict__ lam,
                         float norm, int wb) {
  const int n = ax == 0 ? nx : (ax == 1 ? ny : nz);
  const int n0 = nx * ny * nz, plane = nx * ny;
  const int nlines = nrep * (n0 / n);
  const int lb = (int)((long)blockIdx.x * nlines / gridDim.x);
  const int le = (int)((long)(blockIdx.x + 1) * nlines / gridDim.x);
  // the block's lines in batches of at most wb (the tiles hold n x dst_wpad(wb) floats)
  for (int l0 = lb; l0 < le; l0 += wb) {
  if (l0 > lb) __syncthreads();   // the previous batch's store has read the tiles
  const int W = min(wb, le - l0), Wp = dst_wpad(W);
  const int stride = ax == 0 ? 1 : (ax == 1 ? nx : plane);
  const int tot = W * n;
  // first element of each of this block's lines (and, for the scaling, lx[kx] + ly[ky])
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    const int l = l0 + w;
    int b;
    if (ax == 0) {
      b = l * nx;
    } else if (ax == 1) {
      const int q = l / nx;
      b = q * plane + (l - q * nx);
    } else {
      const int q = l / plane;
      b = q * n0 + (l - q * plane);
    }
    lbase[w] = b;
    if (scale) {
      const int yx = l - (l / plane) * plane;
      const int ky = yx / nx, kx = yx - ky * nx;
      lxy[w] = lam[kx] + lam[nx + ky];
    }
  }
  __syncthreads();
  // e = q D + r over [0, total), stepping by the block size
  auto walk_n = [&](int total, int D, auto&& body) {
    int q = threadIdx.x / D, r = threadIdx.x - q * D;
    const int dq = blockDim.x / D, dr = blockDim.x - dq * D;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      body(e, q, r);
      q += dq;
      r += dr;
      if (r >= D) {
        r -= D;
        ++q;
      }
    }
  };
  auto walk = [&](int D, auto&& body) { walk_n(tot, D, body); };
  // float input: asynchronous 4-byte copies into the tile (all of a thread's loads in flight
  // at once, one wait); float64 input: loads converted to float32
  auto put = [&](float* dst, const VI* src) {
    if constexpr (sizeof(VI) == 4)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr_f(dst)), "l"(src)
                   : "memory");
    else
      *dst = (float)*src;
  };
  if (ax == 0)   // lines are rows: the block's rows are one contiguous range (w = q, k = r)
    walk(n, [&](int e, int w, int k) { put(tA + k * Wp + w, in + l0 * nx + e); });
  else           // element k of consecutive lines: consecutive x (k = q, w = r)
    walk(W, [&](int, int k, int w) { put(tA + k * Wp + w, in + lbase[w] + k * stride); });
  if (Wp > W)   // zero columns past the block's lines
    walk_n(n * (Wp - W), Wp - W, [&](int, int k, int w) { tA[k * Wp + W + w] = 0.0f; });
  if constexpr (sizeof(VI) == 4) asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // src -> dst with m16n8k8 TF32 MMAs: D[i][w] = sum_k A[i][k] B[k][w], A = Se or So
  // (shared, TF32 already), B[k][w] = P_k = x_k + x_{n-1-k} (the middle point of an odd line
  // alone) or M_k = x_k - x_{n-1-k}, formed while the B fragments are loaded.  Each warp takes
  // one 8-line column tile and one parity and forms both of its 16-row output tiles (two
  // independent accumulator chains sharing the B fragments).
  const int hp = (n + 1) >> 1, h = n >> 1;
  const float* Se = S;
  const float* So = S + dst_arows(hp) * dst_astride(hp);
  const int ase = dst_astride(hp), aso = dst_astride(h);
  const int nmte = (hp + 15) >> 4, nmto = (h + 15) >> 4, nnt = Wp >> 3;
  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  auto transform = [&](const float* src, float* dst) {
    for (int task = threadIdx.x >> 5; task < 2 * nnt; task += blockDim.x >> 5) {
      const int odd = task >= nnt;
      const int nt = odd ? task - nnt : task;
      const float* A = odd ? So : Se;
      const int as = odd ? aso : ase, kn = odd ? h : hp, nmt = odd ? nmto : nmte;
      const int col = nt * 8 + gq;
      for (int mp = 0; mp < nmt; mp += 2) {   // output tiles mp, mp + 1 (one pass for n <= 64)
      float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
      for (int k0 = 0; k0 < kn; k0 += 8) {
        uint32_t b[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          // past kn the A columns are zero: any row in the tile will do
          const int k = k0 + tq + 4 * u;
          const int ka = min(k, n - 1), kb = max(n - 1 - k, 0);
          const float xa = src[ka * Wp + col], xb = src[kb * Wp + col];
          const float v = (ka == kb) ? xa : (odd ? xa - xb : xa + xb);
          asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(b[u]) : "f"(v));
        }
#pragma unroll
        for (int mi = 0; mi < 2; ++mi) {
          if (mp + mi < nmt) {
            const float* Ar = A + (16 * (mp + mi) + gq) * as + tq + k0;
            const uint32_t a0 = __float_as_uint(Ar[0]), a1 = __float_as_uint(Ar[8 * as]);
            const uint32_t a2 = __float_as_uint(Ar[4]), a3 = __float_as_uint(Ar[8 * as + 4]);
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, "
                "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                : "+f"(d[mi][0]), "+f"(d[mi][1]), "+f"(d[mi][2]), "+f"(d[mi][3])
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b[0]), "r"(b[1]));
          }
        }
      }
      // D rows 16 m + gq (d0, d1) and 16 m + gq + 8 (d2, d3), columns nt*8 + 2 tq, + 1
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int j0 = 2 * (16 * (mp + mi) + gq) + odd, j1 = j0 + 16;
        if (mp + mi < nmt && j0 < n)
          *reinterpret_cast<float2*>(dst + j0 * Wp + nt * 8 + 2 * tq) = make_float2(d[mi][0], d[mi][1]);
        if (mp + mi < nmt && j1 < n)
          *reinterpret_cast<float2*>(dst + j1 * Wp + nt * 8 + 2 * tq) = make_float2(d[mi][2], d[mi][3]);
      }
      }
    }
    __syncthreads();
  };
  transform(tA, tB);
  const float* res = tB;
  if (scale) {
    const float* lz = lam + nx + ny;
    walk(W, [&](int, int k, int w) { tB[k * Wp + w] *= norm / (lxy[w] + lz[k]); });
    __syncthreads();
    transform(tB, tA);
    res = tA;
  }
  if (ax == 0)
    walk(n, [&](int e, int w, int k) { out[l0 * nx + e] = (VO)res[k * Wp + w]; });
  else
    walk(W, [&](int, int k, int w) { out[lbase[w] + k * stride] = (VO)res[k * Wp + w]; });
  }
}

__device__ __forceinline__ float wsum(float v) { return warp_sumf(v); }
__device__ __forceinline__ double wsum(double v) { return warp_sum(v); }

template <typename V>
__device__ __forceinline__ double* pslot(const Args<V>& a, int rep, int s) {
  return a.part + ((long)rep * kSlots + s) * gridDim.x;
}

template <typename V>
__device__ __forceinline__ V dens(const Args<V>& a, int i) {
  if constexpr (sizeof(V) == 4) return a.drho[i];
  else return a.rho[i];
}
template <typename V>
__device__ __forceinline__ V ghost(const Args<V>& a, int k, int n0, int g) {
  if constexpr (sizeof(V) == 4) return a.gf32[k * n0 + g];
  else return a.gf[k * n0 + g];
}

template <typename V>
__global__ void __launch_bounds__(kThreadsC, 1) k_hartree_coop(Args<V> a) {
  extern __shared__ float smem_tail[];
  __shared__ LevelTable T;
  __shared__ double wpart[kMaxDots][kMaxRep][kWarps];   // per-warp partials of one phase
  __shared__ double sc[kSlots][kMaxRep];                // grid-wide sums
  __shared__ double rz_old[kMaxRep], pAp_old[kMaxRep], beta[kMaxRep], alpha[kMaxRep];
  __shared__ double bbv[kMaxRep];
  __shared__ int act[kMaxRep];   // replica still iterating
  __shared__ int act0[kMaxRep];  // replica solved by this launch
  __shared__ int any_act;
  __shared__ int s_tail_local, s_tail_rep;   // block-local tail (see below)
  const int G = gridDim.x;
  const int gstride = G * blockDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned nbar = 0;
#define COOP_BAR()                                                        \
  do {                                                                    \
    if (!grid_barrier(a.bar, (unsigned)G * (++nbar), a.status)) return; \
  } while (0)
  // per-warp partial of dot d for replica rp (whole warp calls)
  auto put = [&](int d, int rp, V v) {
    v = wsum(v);
    if (lane == 0) wpart[d][rp][warp] = (double)v;
  };
  // block partials of dots 0..nd-1 into slots sl[0..nd-1] (fixed order over warps)
  auto flush = [&](int nd, int s0, int s1, int s2, int s3) {
    __syncthreads();
    const int t = threadIdx.x;
    if (t < nd * a.nrep) {
      const int d = t / a.nrep, rp = t - d * a.nrep;
      const int s = d == 0 ? s0 : d == 1 ? s1 : d == 2 ? s2 : s3;
      double acc = 0.0;
      for (int w = 0; w < kWarps; ++w) acc += wpart[d][rp][w];
      pslot(a, rp, s)[blockIdx.x] = acc;
    }
  };
  // grid-wide sums of slots s0..s(ns-1) into sc (every block, same order)
  auto gsum = [&](int ns, int s0, int s1, int s2, int s3) {
    for (int q = warp; q < ns * a.nrep; q += kWarps) {
      const int k = q / a.nrep, rp = q - k * a.nrep;
      const int s = k == 0 ? s0 : k == 1 ? s1 : k == 2 ? s2 : s3;
      const double* src = pslot(a, rp, s);
      double acc = 0.0;
      for (int b = lane; b < G; b += 32) acc += src[b];
      acc = warp_sum(acc);
      if (lane == 0) sc[s][rp] = acc;
    }
    __syncthreads();
  };

  // flattened quad loops (float path, vec4 with n0 % 128 == 0): the 32 quads of a warp are
  // 128 consecutive points of one replica, so a warp-uniform replica index accumulates the
  // warp's sums of each loop iteration into its own wpart slots
  auto zero_parts = [&](int nd) {
    if (lane == 0)
      for (int d = 0; d < nd; ++d)
        for (int rp = 0; rp < a.nrep; ++rp) wpart[d][rp][warp] = 0.0;
  };
  auto add_part = [&](int d, int rp, float v) {
    v = warp_sumf(v);
    if (lane == 0) wpart[d][rp][warp] += (double)v;
  };

  {  // level table into shared memory
    const int* src = reinterpret_cast<const int*>(a.lt);
    int* dst = reinterpret_cast<int*>(&T);
    for (int i = threadIdx.x; i < (int)(sizeof(LevelTable) / sizeof(int)); i += blockDim.x)
      dst[i] = src[i];
  }
  const int nrep = a.nrep;
  if (threadIdx.x < kMaxRep) {
    act[threadIdx.x] = (threadIdx.x < nrep) && (!a.ctl || a.ctl[threadIdx.x].active);
    act0[threadIdx.x] = act[threadIdx.x];
  }
  __syncthreads();
  const int nl = T.nl, nmulti = T.nmulti;
  const int nx = T.L[0].nx, ny = T.L[0].ny, nz = T.L[0].nz, n0 = T.L[0].n;
  const V ih2 = (V)(1.0 / (a.h * a.h));
  const V hv = (V)a.h;

  // ---- prologue: multipole moments of the density (change) ----------------------------
  bool flat = false;
  if constexpr (sizeof(V) == 4) flat = a.vec4 == 2;
  if (a.mom) {
    // formed by the density kernel: every block sums its per-CTA partials in the same order
    for (int q = warp; q < 4 * nrep; q += kWarps) {
      const int rp = q >> 2, k = q & 3;
      const double* src = a.mom + (long)q * a.nmom;
      double acc = 0.0;
      for (int b = lane; b < a.nmom; b += 32) acc += src[b];
      acc = warp_sum(acc);
      if (lane == 0) sc[4 + k][rp] = acc;
    }
    __syncthreads();
  } else {
  if (flat) {
    if constexpr (sizeof(V) == 4) {
      zero_parts(4);
      if (!a.zero_bc) {
        const int N0 = n0 * nrep;
        const float cx = 0.5f * (float)(nx - 1), cy = 0.5f * (float)(ny - 1);
        const float cz = 0.5f * (float)(nz - 1);
        for (int e0 = 4 * gtid; e0 < N0; e0 += 4 * gstride) {
          const int rp = fdiv(e0, T.L[0].dn);
          if (!act[rp]) continue;
          int ix, iy, iz;
          xyz_of(e0 - rp * n0, nx, ny, T.L[0].dx, T.L[0].dy, ix, iy, iz);
          const float4 v = ld4(a.drho + e0);
          const float s4 = ((v.x + v.y) + v.z) + v.w;
          const float x0 = ((float)ix - cx) * hv;
          const float sx = ((v.x * x0 + v.y * (x0 + hv)) + v.z * (x0 + 2.0f * hv)) +
                           v.w * (x0 + 3.0f * hv);
          add_part(0, rp, s4);
          add_part(1, rp, sx);
          add_part(2, rp, s4 * (((float)iy - cy) * hv));
          add_part(3, rp, s4 * (((float)iz - cz) * hv));
        }
      }
    }
  } else
  for (int rp = 0; rp < nrep; ++rp) {
    V q0 = 0, q1 = 0, q2 = 0, q3 = 0;
    if (act[rp] && !a.zero_bc) {
      for (int g = gtid; g < n0; g += gstride) {
        int ix, iy, iz;
        xyz_of(g, nx, ny, T.L[0].dx, T.L[0].dy, ix, iy, iz);
        const V v = dens(a, rp * n0 + g);
        q0 += v;
        q1 += v * (((V)ix - (V)0.5 * (V)(nx - 1)) * hv);
        q2 += v * (((V)iy - (V)0.5 * (V)(ny - 1)) * hv);
        q3 += v * (((V)iz - (V)0.5 * (V)(nz - 1)) * hv);
      }
    }
    put(0, rp, q0);
    put(1, rp, q1);
    put(2, rp, q2);
    put(3, rp, q3);
  }
  flush(4, 4, 5, 6, 7);
  COOP_BAR();
  gsum(4, 4, 5, 6, 7);
  }

  // ---- right-hand side b = 4 pi rho + ghost term, residual r = b - A x -----------------
  if (flat) {
    if constexpr (sizeof(V) == 4) {
      zero_parts(2);
      const double h3 = a.h * a.h * a.h;
      const int N0 = n0 * nrep;
      for (int e0 = 4 * gtid; e0 < N0; e0 += 4 * gstride) {
        const int rp = fdiv(e0, T.L[0].dn);
        if (!act[rp]) continue;
        const int g0 = e0 - rp * n0;
        int ix, iy, iz;
        xyz_of(g0, nx, ny, T.L[0].dx, T.L[0].dy, ix, iy, iz);
        const float4 dv = ld4(a.drho + e0);
        const float fp = (float)(4.0 * kPi);
        float4 bv = make_float4(fp * dv.x, fp * dv.y, fp * dv.z, fp * dv.w);
        if (!a.zero_bc) {
          const float Q = (float)(h3 * sc[4][rp]), px = (float)(h3 * sc[5][rp]);
          const float py = (float)(h3 * sc[6][rp]), pz = (float)(h3 * sc[7][rp]);
          const float4 g0v = ld4(a.gf32 + g0), g1v = ld4(a.gf32 + n0 + g0);
          const float4 g2v = ld4(a.gf32 + 2 * n0 + g0), g3v = ld4(a.gf32 + 3 * n0 + g0);
          bv.x += Q * g0v.x + px * g1v.x + py * g2v.x + pz * g3v.x;
          bv.y += Q * g0v.y + px * g1v.y + py * g2v.y + pz * g3v.y;
          bv.z += Q * g0v.z + px * g1v.z + py * g2v.z + pz * g3v.z;
          bv.w += Q * g0v.w + px * g1v.w + py * g2v.w + pz * g3v.w;
        }
        float4 xc;
        const float4 ax = A12_quad(a.x + rp * n0, g0, ix, iy, iz, nx, ny, nz, ih2, xc);
        const float4 rv = make_float4(bv.x - ax.x, bv.y - ax.y, bv.z - ax.z, bv.w - ax.w);
        *reinterpret_cast<float4*>(a.r + e0) = rv;
        add_part(0, rp, ((bv.x * bv.x + bv.y * bv.y) + bv.z * bv.z) + bv.w * bv.w);
        add_part(1, rp, ((rv.x * rv.x + rv.y * rv.y) + rv.z * rv.z) + rv.w * rv.w);
      }
    }
  } else {
    const double h3 = a.h * a.h * a.h;
    for (int rp = 0; rp < nrep; ++rp) {
      V bb = 0, rr = 0;
      if (act[rp]) {
        const V Q = (V)(h3 * sc[4][rp]), px = (V)(h3 * sc[5][rp]);
        const V py = (V)(h3 * sc[6][rp]), pz = (V)(h3 * sc[7][rp]);
        const int base = rp * n0;
        for (int g = gtid; g < n0; g += gstride) {
          int ix, iy, iz;
          xyz_of(g, nx, ny, T.L[0].dx, T.L[0].dy, ix, iy, iz);
          V bv = (V)(4.0 * kPi) * dens(a, base + g);
          if (!a.zero_bc)
            bv += Q * ghost(a, 0, n0, g) + px * ghost(a, 1, n0, g) + py * ghost(a, 2, n0, g) +
                  pz * ghost(a, 3, n0, g);
          const V rv = bv - apply_A12<V>(a.x + base, ix, iy, iz, nx, ny, nz, ih2);
          a.r[base + g] = rv;
          bb += bv * bv;
          rr += rv * rv;
        }
      }
      put(0, rp, bb);
      put(1, rp, rr);
    }
  }
  // the coarsest tail level's (transposed) inverse, when small: a shared-memory copy after
  // the tail levels (its load latency overlaps the barrier below; flush syncs the block)
  const float* cinv = a.cinv;
  if (a.dst) {
    // the sine-transform matrices into shared memory (the tiles follow them)
    const int off = dst_mat_floats(nx) + dst_mat_floats(ny) + dst_mat_floats(nz);
    for (int e = threadIdx.x; e < off; e += blockDim.x) smem_tail[e] = a.dst_tab[e];
  } else if (a.cinv && a.cinv_smem && nmulti < nl) {
    int off = 0;
    for (int l = 0; l < T.T.nl; ++l) off += 3 * T.T.n[l];
    const int nc = T.T.n[T.T.nl - 1];
    float* cs = smem_tail + off;
    for (int e = threadIdx.x; e < nc * nc; e += blockDim.x) cs[e] = a.cinv[e];
    cinv = cs;
  }
  flush(2, 0, 1, 0, 0);
  COOP_BAR();
  gsum(2, 0, 1, 0, 0);
  if (threadIdx.x < nrep) {
    const int rp = threadIdx.x;
    bbv[rp] = sc[0][rp];
    if (act[rp] && blockIdx.x == 0) {
      a.st[rp].it = 0;
      a.st[rp].rr = sc[1][rp];
      a.st[rp].status = 0;
    }
  }
  __syncthreads();
  // b = 0: the solution is 0 (CG from a non-zero guess would never meet a relative test)
  for (int rp = 0; rp < nrep; ++rp)
    if (act[rp] && bbv[rp] == 0.0)
      for (int g = gtid; g < n0; g += gstride) a.x[rp * n0 + g] = (V)0;
  __syncthreads();
  if (threadIdx.x < nrep) {
    const int rp = threadIdx.x;
    if (act[rp] && (bbv[rp] == 0.0 || sc[1][rp] <= a.tol * a.tol * bbv[rp])) act[rp] = 0;
  }
  __syncthreads();

  // Blocks whose points of the level above the tail all belong to one replica (that level
  // has at most one point per thread and a multiple of the block size per replica) run the
  // tail of that replica themselves, redundantly, and read its result from shared memory in
  // the first post-sweep above it: no grid barrier and no global round trip in between.
  // (kept in shared memory: s_tail_local, s_tail_rep = -1 for a block without such points)
  if (threadIdx.x == 0) {
    s_tail_local = 0;
    s_tail_rep = -1;
    if (nmulti >= 2 && nmulti < nl) {
      const long na = T.L[nmulti - 1].n;
      if (na % blockDim.x == 0 && na * nrep <= (long)gstride) {
        s_tail_local = 1;
        const long e0 = (long)blockIdx.x * blockDim.x;
        if (e0 < na * nrep) s_tail_rep = (int)(e0 / na);
      }
    }
  }
  __syncthreads();

  int it = 0;
  while (true) {
    if (threadIdx.x == 0) {
      int an = 0;
      for (int rp = 0; rp < nrep; ++rp) an |= act[rp];
      any_act = an;
    }
    __syncthreads();
    if (!any_act) break;

    // ---- sine-transform preconditioner z = M r: five passes, one grid barrier each -------
    if (a.dst) {
      const int wb = a.dst_wb;
      const long tile = (long)max(nx, max(ny, nz)) * dst_wpad(wb);
      const float* Sx = smem_tail;
      const float* Sy = Sx + dst_mat_floats(nx);
      const float* Sz = Sy + dst_mat_floats(ny);
      const int off = dst_mat_floats(nx) + dst_mat_floats(ny) + dst_mat_floats(nz);
      float* tA = smem_tail + off;
      float* tB = tA + ((tile + 3) & ~3L);
      const long wmx = wb;
      int* lbase = reinterpret_cast<int*>(tB + ((tile + 3) & ~3L));
      float* lxy = reinterpret_cast<float*>(lbase + ((wmx + 3) & ~3L));
      const float* lam = a.dst_tab + off;
      const float norm = (float)(8.0 / ((double)(nx + 1) * (ny + 1) * (nz + 1)));
      float* W1 = T.L[0].x;
      float* W2 = T.L[0].t;
      dst_pass<V, float>(0, a.r, W1, nrep, nx, ny, nz, Sx, tA, tB, lbase, lxy, false, lam, norm, wb);
      COOP_BAR();
      dst_pass<float, float>(1, W1, W2, nrep, nx, ny, nz, Sy, tA, tB, lbase, lxy, false, lam, norm, wb);
      COOP_BAR();
      dst_pass<float, float>(2, W2, W1, nrep, nx, ny, nz, Sz, tA, tB, lbase, lxy, true, lam, norm, wb);
      COOP_BAR();
      dst_pass<float, float>(1, W1, W2, nrep, nx, ny, nz, Sy, tA, tB, lbase, lxy, false, lam, norm, wb);
      COOP_BAR();
      dst_pass<float, V>(0, W2, a.z, nrep, nx, ny, nz, Sx, tA, tB, lbase, lxy, false, lam, norm, wb);
      COOP_BAR();
    } else {
    // ---- V-cycle z = M r: down leg over the multi-block levels --------------------------
    for (int l = 0; l < nmulti; ++l) {
      const Level& L = T.L[l];
      const int Nl = L.n * nrep;
      const float ih2f = 1.0f / L.h2, c = kJacobiW * L.h2 / 6.0f;
      if (l == nl - 1) {
        // coarsest level without a tail: damped-Jacobi sweeps from zero, X <-> T
        for (int sw = 0; sw < kCoarseSweeps; ++sw) {
          const float* in = (sw & 1) ? L.t : L.x;
          float* out = (sw & 1) ? L.x : L.t;
          for (int e = gtid; e < Nl; e += gstride) {
            const int rep = fdiv(e, L.dn);
            if (!act[rep]) continue;
            float bv;
            if (l == 0) {
              bv = (float)a.r[e];
              if (sw == 0) L.b[e] = bv;
            } else {
              bv = L.b[e];
            }
            float v;
            if (sw == 0) {
              v = c * bv;
            } else {
              int ix, iy, iz;
              xyz_of(e - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
              float cc;
              const float ax = lap7f(in + rep * L.n, ix, iy, iz, L.nx, L.ny, L.nz, &cc) * ih2f;
              v = cc + c * (bv - ax);
            }
            out[e] = v;
          }
          COOP_BAR();
        }
        if (kCoarseSweeps & 1) {
          for (int e = gtid; e < Nl; e += gstride) L.x[e] = L.t[e];
          COOP_BAR();
        }
        continue;
      }
      // two pre-sweeps from zero in one pass: x = c (2 b - c A b); level 0 reads b from r
      bool pre_done = false;
      if constexpr (sizeof(V) == 4) {
        if (l == 0 && a.vec4) {
          for (int e0 = 4 * gtid; e0 < Nl; e0 += 4 * gstride) {
            const int rep = fdiv(e0, L.dn);
            if (!act[rep]) continue;
            int ix, iy, iz;
            xyz_of(e0 - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
            float4 bc;
            const float4 ab = lap7_quad(a.r + rep * L.n, e0 - rep * L.n, ix, iy, iz, L.nx, L.ny,
                                        L.nz, bc);
            // (no float copy of b = r: the float path's later level-0 passes read r itself)
            *reinterpret_cast<float4*>(L.x + e0) =
                make_float4(c * (2.0f * bc.x - c * ab.x * ih2f), c * (2.0f * bc.y - c * ab.y * ih2f),
                            c * (2.0f * bc.z - c * ab.z * ih2f), c * (2.0f * bc.w - c * ab.w * ih2f));
          }
          pre_done = true;
        }
      }
      if (!pre_done)
      for (int e = gtid; e < Nl; e += gstride) {
        const int rep = fdiv(e, L.dn);
        if (!act[rep]) continue;
        int ix, iy, iz;
        xyz_of(e - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
        const int plane = L.nx * L.ny;
        float bc, sn = 0.0f;
        if (l == 0) {
          const V* rr = a.r;
          bc = (float)rr[e];
          if (ix + 1 < L.nx) sn += (float)rr[e + 1];
          if (ix > 0) sn += (float)rr[e - 1];
          if (iy + 1 < L.ny) sn += (float)rr[e + L.nx];
          if (iy > 0) sn += (float)rr[e - L.nx];
          if (iz + 1 < L.nz) sn += (float)rr[e + plane];
          if (iz > 0) sn += (float)rr[e - plane];
          L.b[e] = bc;
        } else {
          const float* bb = L.b;
          bc = bb[e];
          if (ix + 1 < L.nx) sn += bb[e + 1];
          if (ix > 0) sn += bb[e - 1];
          if (iy + 1 < L.ny) sn += bb[e + L.nx];
          if (iy > 0) sn += bb[e - L.nx];
          if (iz + 1 < L.nz) sn += bb[e + plane];
          if (iz > 0) sn += bb[e - plane];
        }
        L.x[e] = c * (2.0f * bc - c * (6.0f * bc - sn) * ih2f);
      }
      COOP_BAR();
      // residual b - A x of the 8 children of every coarse point, averaged (the box
      // restriction) into the next level's right-hand side, in one pass
      {
        const Level& C = T.L[l + 1];
        const int Nc = C.n * nrep;
        for (int e = gtid; e < Nc; e += gstride) {
          const int rep = fdiv(e, C.dn);
          if (!act[rep]) continue;
          int I, J, K;
          xyz_of(e - rep * C.n, C.nx, C.ny, C.dx, C.dy, I, J, K);
          const float* lb = L.b + rep * L.n;
          if constexpr (sizeof(V) == 4)
            if (l == 0 && a.vec4) lb = a.r + rep * L.n;   // b of level 0 is r
          C.b[e] = restrict_residual(L.x + rep * L.n, lb, I, J, K, L.nx, L.ny, L.nz, ih2f);
        }
      }
      COOP_BAR();
    }
    // ---- tail levels: one block per replica, or every block its own replica's -----------
    if (nmulti < nl) {
      const Level& Lt = T.L[nmulti];
      const bool loc = s_tail_local;
      const int r0 = loc ? (s_tail_rep >= 0 ? s_tail_rep : nrep) : blockIdx.x;
      const int r1 = loc ? r0 + 1 : nrep;
      for (int rp = r0; rp < r1; rp += G)
        if (act[rp])
          tail_vcycle(T.T, Lt.b + rp * Lt.n, loc ? nullptr : Lt.x + rp * Lt.n, cinv, smem_tail);
      if (!loc) COOP_BAR();
    }
    // ---- up leg: x += P x_coarse, two post-sweeps (the last one writes z) ---------------
    for (int l = min(nmulti, nl - 1) - 1; l >= 0; --l) {
      const Level& L = T.L[l];
      const Level& C = T.L[l + 1];
      const int Nl = L.n * nrep;
      const float ih2f = 1.0f / L.h2, c = kJacobiW * L.h2 / 6.0f;
      if (l > 0) {
        // coarse levels: the first post-sweep forms the corrected x = x + P x_coarse of the
        // point and its six neighbours on the fly (one pass, one barrier fewer)
        for (int e = gtid; e < Nl; e += gstride) {
          const int rep = fdiv(e, L.dn);
          if (!act[rep]) continue;
          int ix, iy, iz;
          xyz_of(e - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
          const float* xr = L.x + rep * L.n;
          // (a block-local tail holds this point's replica: rep == s_tail_rep)
          const float* xc = (s_tail_local && l == nmulti - 1) ? smem_tail : C.x + rep * C.n;
          const int g = e - rep * L.n, plane = L.nx * L.ny;
          auto corr = [&](int qx, int qy, int qz, int q) {
            return xr[q] + prolong_point(xc, qx, qy, qz, C.nx, C.ny, C.nz);
          };
          const float c0 = corr(ix, iy, iz, g);
          float sn = 0.0f;
          if (ix + 1 < L.nx) sn += corr(ix + 1, iy, iz, g + 1);
          if (ix > 0) sn += corr(ix - 1, iy, iz, g - 1);
          if (iy + 1 < L.ny) sn += corr(ix, iy + 1, iz, g + L.nx);
          if (iy > 0) sn += corr(ix, iy - 1, iz, g - L.nx);
          if (iz + 1 < L.nz) sn += corr(ix, iy, iz + 1, g + plane);
          if (iz > 0) sn += corr(ix, iy, iz - 1, g - plane);
          L.t[e] = c0 + c * (L.b[e] - (6.0f * c0 - sn) * ih2f);
        }
        COOP_BAR();
      } else {
        bool pdone = false;
        if constexpr (sizeof(V) == 4) {
          if (a.vec4) {
            for (int e0 = 4 * gtid; e0 < Nl; e0 += 4 * gstride) {
              const int rep = fdiv(e0, L.dn);
              if (!act[rep]) continue;
              int ix, iy, iz;
              xyz_of(e0 - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
              const float4 pq = prolong_quad(C.x + rep * C.n, ix, iy, iz, C.nx, C.ny, C.nz);
              float4 v = ld4(L.x + e0);
              v.x += pq.x;
              v.y += pq.y;
              v.z += pq.z;
              v.w += pq.w;
              *reinterpret_cast<float4*>(L.x + e0) = v;
            }
            pdone = true;
          }
        }
        if (!pdone)
          for (int e = gtid; e < Nl; e += gstride) {
            const int rep = fdiv(e, L.dn);
            if (!act[rep]) continue;
            int ix, iy, iz;
            xyz_of(e - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
            L.x[e] += prolong_point(C.x + rep * C.n, ix, iy, iz, C.nx, C.ny, C.nz);
          }
        COOP_BAR();
        bool done = false;
        if constexpr (sizeof(V) == 4) {
          if (a.vec4) {
            for (int e0 = 4 * gtid; e0 < Nl; e0 += 4 * gstride) {
              const int rep = fdiv(e0, L.dn);
              if (!act[rep]) continue;
              int ix, iy, iz;
              xyz_of(e0 - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
              float4 cc;
              const float4 ax = lap7_quad(L.x + rep * L.n, e0 - rep * L.n, ix, iy, iz, L.nx,
                                          L.ny, L.nz, cc);
              const float4 bv = ld4(a.r + e0);   // b of level 0 is r
              *reinterpret_cast<float4*>(L.t + e0) = make_float4(
                  cc.x + c * (bv.x - ax.x * ih2f), cc.y + c * (bv.y - ax.y * ih2f),
                  cc.z + c * (bv.z - ax.z * ih2f), cc.w + c * (bv.w - ax.w * ih2f));
            }
            done = true;
          }
        }
        if (!done)
          for (int e = gtid; e < Nl; e += gstride) {
            const int rep = fdiv(e, L.dn);
            if (!act[rep]) continue;
            int ix, iy, iz;
            xyz_of(e - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
            float cc;
            const float ax = lap7f(L.x + rep * L.n, ix, iy, iz, L.nx, L.ny, L.nz, &cc) * ih2f;
            L.t[e] = cc + c * (L.b[e] - ax);
          }
        COOP_BAR();
      }
      bool done_z = false;
      if constexpr (sizeof(V) == 4) {
        if (l == 0 && a.vec4) {
          for (int e0 = 4 * gtid; e0 < Nl; e0 += 4 * gstride) {
            const int rep = fdiv(e0, L.dn);
            if (!act[rep]) continue;
            int ix, iy, iz;
            xyz_of(e0 - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
            float4 cc;
            const float4 ax = lap7_quad(L.t + rep * L.n, e0 - rep * L.n, ix, iy, iz, L.nx, L.ny,
                                        L.nz, cc);
            const float4 bv = ld4(a.r + e0);   // b of level 0 is r
            *reinterpret_cast<float4*>(a.z + e0) = make_float4(
                cc.x + c * (bv.x - ax.x * ih2f), cc.y + c * (bv.y - ax.y * ih2f),
                cc.z + c * (bv.z - ax.z * ih2f), cc.w + c * (bv.w - ax.w * ih2f));
          }
          done_z = true;
        }
      }
      if (!done_z)
      for (int e = gtid; e < Nl; e += gstride) {
        const int rep = fdiv(e, L.dn);
        if (!act[rep]) continue;
        int ix, iy, iz;
        xyz_of(e - rep * L.n, L.nx, L.ny, L.dx, L.dy, ix, iy, iz);
        float cc;
        const float ax = lap7f(L.t + rep * L.n, ix, iy, iz, L.nx, L.ny, L.nz, &cc) * ih2f;
        const float v = cc + c * (L.b[e] - ax);
        if (l == 0)
          a.z[e] = (V)v;
        else
          L.x[e] = v;
      }
      COOP_BAR();
    }
    if (nl == 1) {  // the fine level is the coarsest: z = its sweeps' result
      const int N0 = n0 * nrep;
      for (int e = gtid; e < N0; e += gstride)
        if (act[fdiv(e, T.L[0].dn)]) a.z[e] = (V)T.L[0].x[e];
      COOP_BAR();
    }
    }   // V-cycle

    // ---- A z and the dot products (r,z), (z,Az), (z,Ap_old), (p_old,Az) ------------------
    const bool first = (it == 0);
    if (flat) {
      if constexpr (sizeof(V) == 4) {
        zero_parts(4);
        const int N0 = n0 * nrep;
        for (int e0 = 4 * gtid; e0 < N0; e0 += 4 * gstride) {
          const int rp = fdiv(e0, T.L[0].dn);
          if (!act[rp]) continue;
          const int g0 = e0 - rp * n0;
          int ix, iy, iz;
          xyz_of(g0, nx, ny, T.L[0].dx, T.L[0].dy, ix, iy, iz);
          float4 zc;
          const float4 az = A12_quad(a.z + rp * n0, g0, ix, iy, iz, nx, ny, nz, ih2, zc);
          *reinterpret_cast<float4*>(a.Az + e0) = az;
          const float4 rv = ld4(a.r + e0);
          add_part(0, rp, ((rv.x * zc.x + rv.y * zc.y) + rv.z * zc.z) + rv.w * zc.w);
          add_part(1, rp, ((zc.x * az.x + zc.y * az.y) + zc.z * az.z) + zc.w * az.w);
          if (!first) {
            const float4 apv = ld4(a.Ap + e0), pv = ld4(a.p + e0);
            add_part(2, rp, ((zc.x * apv.x + zc.y * apv.y) + zc.z * apv.z) + zc.w * apv.w);
            add_part(3, rp, ((pv.x * az.x + pv.y * az.y) + pv.z * az.z) + pv.w * az.w);
          }
        }
      }
    } else
    for (int rp = 0; rp < nrep; ++rp) {
      V d0 = 0, d1 = 0, d2 = 0, d3 = 0;
      bool quads = false;
      if constexpr (sizeof(V) == 4) quads = a.vec4 != 0;
      if (act[rp] && quads) {
        if constexpr (sizeof(V) == 4) {
          const int base = rp * n0;
          const float* zr = a.z + base;
          for (int g0 = 4 * gtid; g0 < n0; g0 += 4 * gstride) {
            int ix, iy, iz;
            xyz_of(g0, nx, ny, T.L[0].dx, T.L[0].dy, ix, iy, iz);
            float4 zc;
            const float4 az = A12_quad(zr, g0, ix, iy, iz, nx, ny, nz, ih2, zc);
            *reinterpret_cast<float4*>(a.Az + base + g0) = az;
            const float4 rv = ld4(a.r + base + g0);
            d0 += rv.x * zc.x;
            d0 += rv.y * zc.y;
            d0 += rv.z * zc.z;
            d0 += rv.w * zc.w;
            d1 += zc.x * az.x;
            d1 += zc.y * az.y;
            d1 += zc.z * az.z;
            d1 += zc.w * az.w;
            if (!first) {
              const float4 apv = ld4(a.Ap + base + g0), pv = ld4(a.p + base + g0);
              d2 += zc.x * apv.x;
              d2 += zc.y * apv.y;
              d2 += zc.z * apv.z;
              d2 += zc.w * apv.w;
              d3 += pv.x * az.x;
              d3 += pv.y * az.y;
              d3 += pv.z * az.z;
              d3 += pv.w * az.w;
            }
          }
        }
      } else if (act[rp]) {
        const int base = rp * n0;
        const V* zr = a.z + base;
        for (int g = gtid; g < n0; g += gstride) {
          int ix, iy, iz;
          xyz_of(g, nx, ny, T.L[0].dx, T.L[0].dy, ix, iy, iz);
          const V zc = zr[g];
          const V az = apply_A12<V>(zr, ix, iy, iz, nx, ny, nz, ih2);
          a.Az[base + g] = az;
          d0 += a.r[base + g] * zc;
          d1 += zc * az;
          if (!first) {
            d2 += zc * a.Ap[base + g];
            d3 += a.p[base + g] * az;
          }
        }
      }
      put(0, rp, d0);
      put(1, rp, d1);
      put(2, rp, d2);
      put(3, rp, d3);
    }
    flush(4, 2, 3, 4, 5);
    COOP_BAR();
    gsum(4, 2, 3, 4, 5);
    // beta (Polak-Ribiere), (p, Ap) with p = z + beta p_old, Ap = Az + beta Ap_old, alpha
    if (threadIdx.x < nrep && act[threadIdx.x]) {
      const int rp = threadIdx.x;
      const double rz = sc[2][rp];
      double bt = 0.0, pAp = sc[3][rp];
      if (!first) {
        bt = (rz - sc[6][rp]) / rz_old[rp];
        pAp = sc[3][rp] + bt * (sc[4][rp] + sc[5][rp]) + bt * bt * pAp_old[rp];
      }
      beta[rp] = bt;
      alpha[rp] = rz / pAp;
      rz_old[rp] = rz;
      pAp_old[rp] = pAp;
    }
    __syncthreads();

    // ---- p, Ap, x, r updates; partials of (r,r) and (r_new, z_old) ----------------------
    if (flat) {
      if constexpr (sizeof(V) == 4) {
        zero_parts(2);
        const int N0 = n0 * nrep;
        for (int e = 4 * gtid; e < N0; e += 4 * gstride) {
          const int rp = fdiv(e, T.L[0].dn);
          if (!act[rp]) continue;
          const float al = (float)alpha[rp], bt = (float)beta[rp];
          const float4 zc = ld4(a.z + e), az = ld4(a.Az + e), xv = ld4(a.x + e),
                       rv = ld4(a.r + e);
          float4 pv = zc, apv = az;
          if (!first) {
            const float4 po = ld4(a.p + e), apo = ld4(a.Ap + e);
            pv = make_float4(fmaf(bt, po.x, zc.x), fmaf(bt, po.y, zc.y), fmaf(bt, po.z, zc.z),
                             fmaf(bt, po.w, zc.w));
            apv = make_float4(fmaf(bt, apo.x, az.x), fmaf(bt, apo.y, az.y),
                              fmaf(bt, apo.z, az.z), fmaf(bt, apo.w, az.w));
          }
          const float4 rn = make_float4(fmaf(-al, apv.x, rv.x), fmaf(-al, apv.y, rv.y),
                                        fmaf(-al, apv.z, rv.z), fmaf(-al, apv.w, rv.w));
          *reinterpret_cast<float4*>(a.p + e) = pv;
          *reinterpret_cast<float4*>(a.Ap + e) = apv;
          *reinterpret_cast<float4*>(a.x + e) =
              make_float4(fmaf(al, pv.x, xv.x), fmaf(al, pv.y, xv.y), fmaf(al, pv.z, xv.z),
                          fmaf(al, pv.w, xv.w));
          *reinterpret_cast<float4*>(a.r + e) = rn;
          add_part(0, rp, ((rn.x * rn.x + rn.y * rn.y) + rn.z * rn.z) + rn.w * rn.w);
          add_part(1, rp, ((rn.x * zc.x + rn.y * zc.y) + rn.z * zc.z) + rn.w * zc.w);
        }
      }
    } else
    for (int rp = 0; rp < nrep; ++rp) {
      V d0 = 0, d1 = 0;
      bool quads = false;
      if constexpr (sizeof(V) == 4) quads = a.vec4 != 0;
      if (act[rp] && quads) {
        if constexpr (sizeof(V) == 4) {
          const int base = rp * n0;
          const float al = (float)alpha[rp], bt = (float)beta[rp];
          for (int g0 = 4 * gtid; g0 < n0; g0 += 4 * gstride) {
            const int e = base + g0;
            const float4 zc = ld4(a.z + e), az = ld4(a.Az + e), xv = ld4(a.x + e),
                         rv = ld4(a.r + e);
            float4 pv = zc, apv = az;
            if (!first) {
              const float4 po = ld4(a.p + e), apo = ld4(a.Ap + e);
              pv = make_float4(fmaf(bt, po.x, zc.x), fmaf(bt, po.y, zc.y), fmaf(bt, po.z, zc.z),
                               fmaf(bt, po.w, zc.w));
              apv = make_float4(fmaf(bt, apo.x, az.x), fmaf(bt, apo.y, az.y),
                                fmaf(bt, apo.z, az.z), fmaf(bt, apo.w, az.w));
            }
            const float4 xn = make_float4(fmaf(al, pv.x, xv.x), fmaf(al, pv.y, xv.y),
                                          fmaf(al, pv.z, xv.z), fmaf(al, pv.w, xv.w));
            const float4 rn = make_float4(fmaf(-al, apv.x, rv.x), fmaf(-al, apv.y, rv.y),
                                          fmaf(-al, apv.z, rv.z), fmaf(-al, apv.w, rv.w));
            *reinterpret_cast<float4*>(a.p + e) = pv;
            *reinterpret_cast<float4*>(a.Ap + e) = apv;
            *reinterpret_cast<float4*>(a.x + e) = xn;
            *reinterpret_cast<float4*>(a.r + e) = rn;
            d0 += rn.x * rn.x;
            d0 += rn.y * rn.y;
            d0 += rn.z * rn.z;
            d0 += rn.w * rn.w;
            d1 += rn.x * zc.x;
            d1 += rn.y * zc.y;
            d1 += rn.z * zc.z;
            d1 += rn.w * zc.w;
          }
        }
      } else if (act[rp]) {
        const int base = rp * n0;
        const V al = (V)alpha[rp], bt = (V)beta[rp];
        for (int g = gtid; g < n0; g += gstride) {
          const int e = base + g;
          const V zc = a.z[e], az = a.Az[e];
          const V pv = first ? zc : fma(bt, a.p[e], zc);
          const V apv = first ? az : fma(bt, a.Ap[e], az);
          a.p[e] = pv;
          a.Ap[e] = apv;
          a.x[e] = fma(al, pv, a.x[e]);
          const V rv = fma(-al, apv, a.r[e]);
          a.r[e] = rv;
          d0 += rv * rv;
          d1 += rv * zc;
        }
      }
      put(0, rp, d0);
      put(1, rp, d1);
    }
    flush(2, 1, 6, 0, 0);
    COOP_BAR();
    gsum(2, 1, 6, 0, 0);
    ++it;
    if (threadIdx.x < nrep && act[threadIdx.x]) {
      const int rp = threadIdx.x;
      const double rr = sc[1][rp];
      int st = 0;
      if (!(rr <= 1e300)) {
        st = RMGTD_EDIVERGED;
        act[rp] = 0;
      } else if (rr <= a.tol * a.tol * bbv[rp]) {
        act[rp] = 0;
      } else if (it >= a.max_it) {
        st = RMGTD_ENOTCONVERGED;
        act[rp] = 0;
      }
      if (blockIdx.x == 0) {
        if (st) {
          atomicCAS(a.status, 0, st);
          a.st[rp].status = st;
        }
        a.st[rp].it = it;
        a.st[rp].rr = rr;
      }
    }
    __syncthreads();
  }
  if (a.counters && blockIdx.x == 0 && threadIdx.x < nrep && act0[threadIdx.x]) {
    atomicAdd(&a.counters[0], 1ull);
    atomicAdd(&a.counters[1], (unsigned long long)a.st[threadIdx.x].it);
  }
  // closing phase of the mixed pass: the potential change dV = dV_H + dV_xc of every replica
  // solved here (the last barrier published x), in the same arithmetic as k_xc_mixed
  if constexpr (sizeof(V) == 4) {
    if (a.dv_out) {
      const int N0 = n0 * nrep;
      for (int e = gtid; e < N0; e += gstride) {
        const int rp = fdiv(e, T.L[0].dn);
        if (!act0[rp]) continue;
        const int g = e - rp * n0;
        a.dv_out[e] = dvxc_increment(a.rho0 + g, a.rho0f[g], a.drho[e]) + a.x[e];
      }
    }
  }
#undef COOP_BAR
}

}  // namespace coop

// shared memory of the sine-transform preconditioner with batches of wb lines: the three
// matrices, two tiles of n_max x dst_wpad(wb) floats and one int and one float per line
static size_t dst_smem_batch(const rmgtd_ctx* ctx, int wb) {
  const int nmax = std::max(ctx->nx, std::max(ctx->ny, ctx->nz));
  const size_t fl = (size_t)dst_mat_floats(ctx->nx) + dst_mat_floats(ctx->ny) + dst_mat_floats(ctx->nz);
  const size_t tile = (size_t)nmax * dst_wpad(wb);
  return sizeof(float) * (fl + 2 * ((tile + 3) & ~(size_t)3) + 2 * (((size_t)wb + 3) & ~(size_t)3));
}

// lines per batch of a transform pass for a launch of `grid` blocks: every line of a block
// at once when that fits in kDstSmemMax, else the largest batch (at least 8 lines) that does;
// 0 when not even that fits
static int dst_batch_lines(const rmgtd_ctx* ctx, int nrep, int grid) {
  long wmax = 0;
  for (int n : {ctx->nx, ctx->ny, ctx->nz})
    wmax = std::max(wmax, ((long)nrep * ctx->Ng / n + grid - 1) / grid);
  int wb = (int)std::max(1L, wmax);
  while (wb > 8 && dst_smem_batch(ctx, wb) > kDstSmemMax) wb = std::max(8, wb * 3 / 4);
  return dst_smem_batch(ctx, wb) <= kDstSmemMax ? wb : 0;
}

static size_t dst_smem_bytes(const rmgtd_ctx* ctx, int nrep, int grid) {
  const int wb = dst_batch_lines(ctx, nrep, grid);
  return wb > 0 ? dst_smem_batch(ctx, wb) : (size_t)-1;
}

// the preconditioner a solve of all replicas uses (RMGTD_PRECOND_DST when requested and its
// tables and tiles fit in shared memory, else RMGTD_PRECOND_MG)
int hartree_precond_in_use(rmgtd_ctx* ctx) {
  const int kk = ctx->mixed ? 1 : 0;
  const int grid = std::max(1, (ctx->coop_attr_set[kk] ? ctx->coop_grid[kk]
                                                       : std::min(ctx->num_sms, ctx->red_cap)) /
                                   std::max(1, ctx->tune_coop_div));
  const int use_dst = ctx->dst_tab && ctx->hartree_precond == RMGTD_PRECOND_DST &&
                      dst_smem_bytes(ctx, ctx->nrep, grid) <= kDstSmemMax &&
                      (long)ctx->nrep * ctx->Ng < (1L << 31);
  return use_dst ? RMGTD_PRECOND_DST : RMGTD_PRECOND_MG;
}

// host launcher of the persistent solve; f32 selects the mixed-path correction solve
int hartree_coop(rmgtd_ctx* ctx, const double* rho, double* vh, const RepCtl* ctl, int zero_bc,
                 int nrep, int f32, int xc_fuse) {
  if (nrep > coop::kMaxRep) return set_error(ctx, RMGTD_EINVAL, "too many replicas");
  if (f32 && (!ctx->drho32 || !ctx->ghost32))
    return set_error(ctx, RMGTD_ESTATE, "mixed Hartree solve without float32 buffers");
  const int kk = f32 ? 1 : 0;
  const int grid = std::max(1, (ctx->coop_attr_set[kk] ? ctx->coop_grid[kk]
                                                       : std::min(ctx->num_sms, ctx->red_cap)) /
                                   std::max(1, ctx->tune_coop_div));
  size_t smem = ctx->mg_tail_smem;
  const size_t dsm = dst_smem_bytes(ctx, nrep, grid);
  const int use_dst = ctx->dst_tab && ctx->hartree_precond == RMGTD_PRECOND_DST &&
                      dsm <= kDstSmemMax && (long)nrep * ctx->Ng < (1L << 31);
  if (use_dst) smem = std::max(smem, dsm);
  auto fill = [&](auto& a) {
    a.lt = (const LevelTable*)ctx->mg_table;
    a.nrep = nrep;
    a.h = ctx->h;
    a.rho = rho;
    a.drho = ctx->drho32;
    a.gf = ctx->ghost;
    a.gf32 = ctx->ghost32;
    a.cinv = ctx->mg_cinv;
    a.cinv_smem = ctx->mg_cinv_smem;
    a.dst = use_dst;
    a.dst_wb = use_dst ? dst_batch_lines(ctx, nrep, grid) : 0;
    a.dst_tab = ctx->dst_tab;
    a.zero_bc = zero_bc;
    a.part = ctx->red_part;
    a.st = ctx->pcg;
    a.ctl = ctl;
    a.max_it = ctx->opt.poisson_max_iter;
    a.bar = ctx->bar2;
    a.status = ctx->status;
    a.counters = ctx->tune_x ? nullptr : ctx->kexec + 2;
    // quads of the float path (16-byte aligned rows); 2: also warp-uniform replicas
    a.vec4 = (ctx->nx % 4 == 0) ? (((long)ctx->Ng % 128 == 0) ? 2 : 1) : 0;
    a.rho0 = ctx->rho_xc_ref;    // rho_ref (+ the frozen core): the xc increment's base
    a.rho0f = ctx->rho_ref32;
    a.dv_out = nullptr;
    a.mom = nullptr;
    a.nmom = 0;
  };
  const void* fn;
  void* args[1];
  coop::Args<float> af;
  coop::Args<double> ad;
  if (f32) {
    fill(af);
    af.x = ctx->tune_x ? (float*)ctx->tune_x : ctx->dvh32;
    af.r = ctx->pcg32_r;
    af.z = ctx->pcg32_z;
    af.p = ctx->pcg32_p;
    af.Ap = ctx->pcg32_Ap;
    af.Az = ctx->pcg32_Az;
    af.tol = ctx->opt.mixed_poisson_tol > 0.0 ? std::max(ctx->opt.mixed_poisson_tol, 1e-8)
                                              : std::max(ctx->opt.poisson_tol, kMixedPoissonTol);
    if (xc_fuse && !ctx->tune_x && ctx->rho_ref32) af.dv_out = ctx->dv32;
    // the mixed pass: moments from the density kernel that just ran
    if (xc_fuse && !ctx->tune_x && ctx->rho_mom_blocks > 0 && rho == ctx->rho) {
      af.mom = ctx->rho_mom;
      af.nmom = ctx->rho_mom_blocks;
    }
    fn = (const void*)coop::k_hartree_coop<float>;
    args[0] = &af;
  } else {
    fill(ad);
    ad.x = ctx->tune_x ? (double*)ctx->tune_x : vh;
    ad.r = ctx->pcg_r;
    ad.z = ctx->pcg_z;
    ad.p = ctx->pcg_p;
    ad.Ap = ctx->pcg_Ap;
    ad.Az = ctx->pcg_Az;
    ad.tol = ctx->opt.poisson_tol;
    fn = (const void*)coop::k_hartree_coop<double>;
    args[0] = &ad;
  }
  const int k = f32 ? 1 : 0;
  // the shared-memory limit is an attribute of the function, shared by every context of the
  // process: only ever raise it (contexts of other grids may need more or less)
  {
    cudaFuncAttributes fa;
    RMGTD_CUDA(ctx, cudaFuncGetAttributes(&fa, fn));
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
      RMGTD_CUDA(ctx, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
  }
  if (!ctx->coop_attr_set[k]) {
    int per_sm = 0;
    RMGTD_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, coop::kThreadsC, smem));
    if (per_sm < 1) return set_error(ctx, RMGTD_ECUDA, "persistent Hartree kernel does not fit on an SM");
    ctx->coop_grid[k] = std::min(per_sm * ctx->num_sms, ctx->red_cap);
    ctx->coop_attr_set[k] = 1;
  }
  // the tiles of the sine-transform passes were sized for this grid
  if (std::max(1, ctx->coop_grid[k] / std::max(1, ctx->tune_coop_div)) != grid)
    return set_error(ctx, RMGTD_ECUDA, "persistent Hartree grid differs from the planned one");
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->bar2, 0, sizeof(unsigned), ctx->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(coop::kThreadsC);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  RMGTD_CUDA(ctx, cudaLaunchKernelExC(&cfg, fn, args));
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_hartree_coop");
  return RMGTD_OK;
}

// Start of a step in one launch: H_1 <- 2 H_0 - H_-1 and the control blocks reset (as
// k_step_begin) together with the initial guess of the step's first Hartree solve, the
// quadratic extrapolation in time of the last three solutions,
//   x <- 3 x(t) - 3 x(t - dt) + x(t - 2 dt)
// (error O(dt^3) against O(dt^2) for the linear 2 x(t) - x(t - dt)); p2 <- p1, p1 <- x(t).
// Only the CG starting point changes, not the solution it converges to.
template <typename T>
__global__ void k_begin_extrap(long n, const double* __restrict__ H0,
                               const double* __restrict__ Hm1, const double* __restrict__ Hm2,
                               double* __restrict__ H1,
                               RepCtl* ctl, int nrep, const int* __restrict__ failed,
                               int* status, long n2, T* __restrict__ x, T* __restrict__ p1,
                               T* __restrict__ p2) {
  const int f = *failed;
  if (!f) {
    const long stride = (long)gridDim.x * blockDim.x;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += stride)
      H1[e] = Hm2 ? 3.0 * (H0[e] - Hm1[e]) + Hm2[e] : 2.0 * H0[e] - Hm1[e];
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n2; e += stride) {
      const T t = x[e], q = p1[e];
      x[e] = (T)3 * (t - q) + p2[e];
      p2[e] = q;
      p1[e] = t;
    }
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

int step_begin_extrapolate(rmgtd_ctx* ctx) {
  if (!ctx->hartree_xc) return step_begin(ctx);
  const long n = (long)ctx->nrep * ctx->N * ctx->N;
  const long n2 = (long)ctx->nrep * ctx->Ng;
  const int bl = (int)std::max<long>(1, std::min<long>(ceil_div(n2, kThreads), 65535L));
  if (ctx->mixed)
    k_begin_extrap<float><<<bl, kThreads, 0, ctx->stream>>>(
        n, ctx->H0, ctx->Hm1, ctx->Hm2, ctx->H1, ctx->ctl, ctx->nrep, ctx->failed, ctx->status,
        n2, ctx->dvh32, ctx->dvh_prev32, ctx->dvh_prev2_32);
  else
    k_begin_extrap<double><<<bl, kThreads, 0, ctx->stream>>>(
        n, ctx->H0, ctx->Hm1, ctx->Hm2, ctx->H1, ctx->ctl, ctx->nrep, ctx->failed, ctx->status,
        n2, ctx->vh, ctx->vh_prev, ctx->vh_prev2);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_begin_extrap");
  return RMGTD_OK;
}


// no history yet: p1 = p2 = current, so the first extrapolations reproduce the current guess
int hartree_reset_history(rmgtd_ctx* ctx) {
  const long n = (long)ctx->nrep * ctx->Ng;
  for (double* p : {ctx->vh_prev, ctx->vh_prev2})
    RMGTD_CUDA(ctx, cudaMemcpyAsync(p, ctx->vh, sizeof(double) * n, cudaMemcpyDeviceToDevice,
                                    ctx->stream));
  if (ctx->mixed)
    for (float* p : {ctx->dvh_prev32, ctx->dvh_prev2_32})
      RMGTD_CUDA(ctx, cudaMemcpyAsync(p, ctx->dvh32, sizeof(float) * n, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
  return RMGTD_OK;
}

}  // namespace rmgtd
