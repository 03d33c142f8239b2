// Grid operators: local ionic potential, Kleinman-Bylander projectors, H applied to an
// orbital block (Eq. 1 with the 12th-order stencil of Eq. 2), and LDA exchange-correlation.
#include <math.h>

#include "lda.cuh"
#include "rmgtd_internal.cuh"

namespace rmgtd {

// ---------------------------------------------------------------------------------------
// Local potential: sum_a -Z_a erf(r/rc_a)/r (value -2 Z_a/(rc_a sqrt(pi)) at r = 0), plus the
// harmonic test well 0.5 w^2 r^2 when w > 0.
__global__ void k_vion(int nx, int ny, int nz, double h, int natoms,
                       const double* __restrict__ pos, const double* __restrict__ Z,
                       const double* __restrict__ rc, double omega, double* __restrict__ v) {
  const long Ng = (long)nx * ny * nz;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < Ng;
       g += (long)gridDim.x * blockDim.x) {
    const int ix = (int)(g % nx);
    const int iy = (int)((g / nx) % ny);
    const int iz = (int)(g / ((long)nx * ny));
    const double x = axis_coord(ix, nx, h), y = axis_coord(iy, ny, h), z = axis_coord(iz, nz, h);
    double acc = 0.0;
    for (int a = 0; a < natoms; ++a) {
      const double dx = x - pos[3 * a], dy = y - pos[3 * a + 1], dz = z - pos[3 * a + 2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (r > 0.0)
        acc -= Z[a] * erf(r / rc[a]) / r;
      else
        acc -= 2.0 * Z[a] / (rc[a] * 1.7724538509055160273);
    }
    if (omega > 0.0) acc += 0.5 * omega * omega * (x * x + y * y + z * z);
    v[g] = acc;
  }
}

int launch_vion(rmgtd_ctx* ctx, const double* pos, const double* Z, const double* rc,
                int natoms) {
  const int blocks = (int)std::min<long>(ceil_div(ctx->Ng, kThreads), 8L * ctx->num_sms);
  k_vion<<<blocks, kThreads, 0, ctx->stream>>>(ctx->nx, ctx->ny, ctx->nz, ctx->h, natoms, pos,
                                               Z, rc, ctx->v_ext_omega, ctx->vion);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_vion");
  return RMGTD_OK;
}

// ---------------------------------------------------------------------------------------
// Projector values on their boxes: s = exp(-r^2/rc^2), p = (q - R_q) exp(-r^2/rc^2), zero for
// r^2 > 25 rc^2; one block per projector, then normalised to h^3 sum beta^2 = 1.
__global__ void k_proj_values(int nx, int ny, int nz, double h, const int* __restrict__ box,
                              const long long* __restrict__ off,
                              const double* __restrict__ center, const int* __restrict__ lm,
                              const double* __restrict__ prc, double* __restrict__ val) {
  const int p = blockIdx.x;
  const int x0 = box[6 * p], y0 = box[6 * p + 1], z0 = box[6 * p + 2];
  const int bx = box[6 * p + 3], by = box[6 * p + 4], bz = box[6 * p + 5];
  const long nb = (long)bx * by * bz;
  const double R0 = center[3 * p], R1 = center[3 * p + 1], R2 = center[3 * p + 2];
  const double rcp = prc[p];
  const int l = lm[2 * p], m = lm[2 * p + 1];
  double* out = val + off[p];
  __shared__ double sh[32];
  double ss = 0.0;
  for (long e = threadIdx.x; e < nb; e += blockDim.x) {
    const int ix = x0 + (int)(e % bx), iy = y0 + (int)((e / bx) % by), iz = z0 + (int)(e / ((long)bx * by));
    const double dx = axis_coord(ix, nx, h) - R0, dy = axis_coord(iy, ny, h) - R1,
                 dz = axis_coord(iz, nz, h) - R2;
    const double r2 = dx * dx + dy * dy + dz * dz;
    double b = 0.0;
    if (r2 <= 25.0 * rcp * rcp) {
      b = exp(-r2 / (rcp * rcp));
      if (l == 1) b *= (m == 0 ? dx : (m == 1 ? dy : dz));
    }
    out[e] = b;
    ss += b * b;
  }
  ss = block_sum(ss, sh);
  __shared__ double scale;
  if (threadIdx.x == 0) scale = (ss > 0.0) ? 1.0 / sqrt(h * h * h * ss) : 0.0;
  __syncthreads();
  for (long e = threadIdx.x; e < nb; e += blockDim.x) out[e] *= scale;
}

int build_projectors(rmgtd_ctx* ctx, const rmgtd_system* sys) {
  ctx->nproj = sys->nproj;
  if (sys->nproj == 0) return RMGTD_OK;
  const int np = sys->nproj;
  std::vector<int> box(6 * np), lm(2 * np);
  std::vector<long long> off(np + 1, 0);
  std::vector<double> cen(3 * np);
  const int n[3] = {ctx->nx, ctx->ny, ctx->nz};
  for (int p = 0; p < np; ++p) {
    const int a = sys->proj_atom[p];
    if (a < 0 || a >= sys->natoms)
      return set_error(ctx, RMGTD_EINVAL, "proj_atom out of range");
    const double R = 5.0 * sys->proj_rc[p];
    for (int d = 0; d < 3; ++d) {
      const double c = sys->pos[3 * a + d];
      cen[3 * p + d] = c;
      // generous integer bounds; the sphere test inside the kernel decides membership
      int lo = (int)floor((c - R) / ctx->h + 0.5 * (n[d] - 1)) - 1;
      int hi = (int)ceil((c + R) / ctx->h + 0.5 * (n[d] - 1)) + 1;
      lo = std::max(lo, 0);
      hi = std::min(hi, n[d] - 1);
      if (hi < lo) { lo = 0; hi = -1; }
      box[6 * p + d] = lo;
      box[6 * p + 3 + d] = std::max(hi - lo + 1, 0);
    }
    const long long nb = (long long)box[6 * p + 3] * box[6 * p + 4] * box[6 * p + 5];
    off[p + 1] = off[p] + nb;
    lm[2 * p] = sys->proj_l[p];
    lm[2 * p + 1] = sys->proj_m ? sys->proj_m[p] : 0;
    if (lm[2 * p] < 0 || lm[2 * p] > 1 || lm[2 * p + 1] < 0 || lm[2 * p + 1] > 2)
      return set_error(ctx, RMGTD_EINVAL, "projector l must be 0 or 1 and m in 0..2");
  }
  ctx->h_pbox = box;
  ctx->h_poff = off;
  ctx->h_Ekb.assign(sys->E_kb, sys->E_kb + np);
  ctx->pbox = (int*)dev_alloc(ctx, sizeof(int) * 6 * np);
  ctx->poff = (long long*)dev_alloc(ctx, sizeof(long long) * (np + 1));
  ctx->pval = (double*)dev_alloc(ctx, sizeof(double) * std::max<long long>(off[np], 1));
  ctx->Ekb = (double*)dev_alloc(ctx, sizeof(double) * np);
  int* lm_d = (int*)dev_alloc(ctx, sizeof(int) * 2 * np);
  double* cen_d = (double*)dev_alloc(ctx, sizeof(double) * 3 * np);
  double* rc_d = (double*)dev_alloc(ctx, sizeof(double) * np);
  if (!ctx->pbox || !ctx->poff || !ctx->pval || !ctx->Ekb || !lm_d || !cen_d || !rc_d)
    return set_error(ctx, RMGTD_ENOMEM, "projector allocation failed");
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->pbox, box.data(), sizeof(int) * 6 * np,
                                  cudaMemcpyHostToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->poff, off.data(), sizeof(long long) * (np + 1),
                                  cudaMemcpyHostToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Ekb, sys->E_kb, sizeof(double) * np,
                                  cudaMemcpyHostToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(lm_d, lm.data(), sizeof(int) * 2 * np,
                                  cudaMemcpyHostToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(cen_d, cen.data(), sizeof(double) * 3 * np,
                                  cudaMemcpyHostToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(rc_d, sys->proj_rc, sizeof(double) * np,
                                  cudaMemcpyHostToDevice, ctx->stream));
  k_proj_values<<<np, kThreads, 0, ctx->stream>>>(ctx->nx, ctx->ny, ctx->nz, ctx->h, ctx->pbox,
                                                  ctx->poff, cen_d, lm_d, rc_d, ctx->pval);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_proj_values");
  RMGTD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return RMGTD_OK;
}

// ---------------------------------------------------------------------------------------
// Element-type helpers for the templated stencil (real / interleaved complex).
template <typename T> struct Elem;
template <> struct Elem<double> { typedef double S; };
template <> struct Elem<float> { typedef float S; };
template <> struct Elem<double2> { typedef double S; };
template <> struct Elem<float2> { typedef float S; };

__device__ __forceinline__ double zero_of(double) { return 0.0; }
__device__ __forceinline__ float zero_of(float) { return 0.0f; }
__device__ __forceinline__ double2 zero_of(double2) { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float2 zero_of(float2) { return make_float2(0.0f, 0.0f); }
__device__ __forceinline__ double fmac(double c, double x, double a) { return fma(c, x, a); }
__device__ __forceinline__ float fmac(float c, float x, float a) { return fmaf(c, x, a); }
__device__ __forceinline__ double2 fmac(double c, double2 x, double2 a) {
  return make_double2(fma(c, x.x, a.x), fma(c, x.y, a.y));
}
__device__ __forceinline__ float2 fmac(float c, float2 x, float2 a) {
  return make_float2(fmaf(c, x.x, a.x), fmaf(c, x.y, a.y));
}
__device__ __forceinline__ double add2(double a, double b) { return a + b; }
__device__ __forceinline__ float add2(float a, float b) { return a + b; }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double dot_re(double a, double b) { return a * b; }
__device__ __forceinline__ double dot_re(float a, float b) { return (double)a * (double)b; }

// out = cscale * Lap_12(x) * h^2 + v * x  with cscale = -1/(2 h^2): H x without the KB part.
// Block BX x BY threads over an x-y tile; each thread marches along z through `zchunk`
// planes keeping its z-column in registers; the x-y neighbourhood of each plane is staged in
// shared memory with a 6-point halo.  Ghost values outside the grid are zero.
template <typename T, int BX, int BY>
__global__ void __launch_bounds__(BX * BY)
k_hstencil(const T* __restrict__ x, T* __restrict__ out, const double* __restrict__ v0,
           const double* __restrict__ v1, int nx, int ny, int nz, int zchunk, int nzc,
           double cscale, long Ng) {
  typedef typename Elem<T>::S S;
  constexpr int R = kFdRadius;
  constexpr int TX = BX + 2 * R, TY = BY + 2 * R;
  __shared__ T tile[TY][TX];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * BX + tx;
  const int col = blockIdx.z / nzc;
  const int z0 = (blockIdx.z % nzc) * zchunk;
  const int z1 = min(nz, z0 + zchunk);
  const int ix = blockIdx.x * BX + tx, iy = blockIdx.y * BY + ty;
  const bool in_xy = (ix < nx) && (iy < ny);
  const T* xc = x + (long)col * Ng;
  T* oc = out + (long)col * Ng;
  const long plane = (long)nx * ny;
  S c[R + 1];
#pragma unroll
  for (int m = 0; m <= R; ++m) c[m] = (S)(fd_coef(m) * cscale);
  const S c0 = (S)(3.0 * fd_coef(0) * cscale);
  T q[2 * R + 1];
#pragma unroll
  for (int k = 0; k < 2 * R; ++k) {
    const int z = z0 - R + k;
    q[k] = (in_xy && z >= 0 && z < nz) ? xc[(long)z * plane + (long)iy * nx + ix] : zero_of(T());
  }
  for (int z = z0; z < z1; ++z) {
    {
      const int zz = z + R;
      q[2 * R] = (in_xy && zz < nz) ? xc[(long)zz * plane + (long)iy * nx + ix] : zero_of(T());
    }
    // stage the x-y plane with its halo
    for (int e = tid; e < TX * TY; e += BX * BY) {
      const int ly = e / TX, lx = e % TX;
      const int gx = blockIdx.x * BX + lx - R, gy = blockIdx.y * BY + ly - R;
      const bool corner = (lx < R || lx >= BX + R) && (ly < R || ly >= BY + R);
      T val = zero_of(T());
      if (!corner && gx >= 0 && gx < nx && gy >= 0 && gy < ny)
        val = xc[(long)z * plane + (long)gy * nx + gx];
      tile[ly][lx] = val;
    }
    __syncthreads();
    if (in_xy) {
      const T ctr = q[R];
      T acc = fmac(c0, ctr, zero_of(T()));
#pragma unroll
      for (int m = 1; m <= R; ++m) {
        T s = add2(add2(tile[ty + R][tx + R + m], tile[ty + R][tx + R - m]),
                   add2(tile[ty + R + m][tx + R], tile[ty + R - m][tx + R]));
        s = add2(s, add2(q[R + m], q[R - m]));
        acc = fmac(c[m], s, acc);
      }
      const long g = (long)z * plane + (long)iy * nx + ix;
      double vv = v0[g];
      if (v1) vv += v1[g];
      oc[g] = fmac((S)vv, ctr, acc);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2 * R; ++k) q[k] = q[k + 1];
  }
}

// KB projections c[p][j] = h^3 sum_box beta_p x_j (one block per (p, j); complex parts
// handled as two real sums).
template <typename T>
__global__ void k_kb_project(const T* __restrict__ x, int ncols, long Ng, int nx, int ny,
                             const int* __restrict__ box, const long long* __restrict__ off,
                             const double* __restrict__ val, double h3, double* __restrict__ coef) {
  const int p = blockIdx.x, j = blockIdx.y;
  const int x0 = box[6 * p], y0 = box[6 * p + 1], z0 = box[6 * p + 2];
  const int bx = box[6 * p + 3], by = box[6 * p + 4], bz = box[6 * p + 5];
  const int nb = bx * by * bz, bxy = bx * by;   // a box holds fewer than 2^31 points
  const double* b = val + off[p];
  const T* xc = x + (long)j * Ng;
  __shared__ double sh[32];
  double sr = 0.0, si = 0.0;
  for (int e = threadIdx.x; e < nb; e += blockDim.x) {
    const int ez = e / bxy, exy = e - ez * bxy, ey = exy / bx, ex = exy - ey * bx;
    const long g = ((long)(z0 + ez) * ny + (y0 + ey)) * nx + x0 + ex;
    const T xv = xc[g];
    if constexpr (sizeof(T) == 2 * sizeof(typename Elem<T>::S)) {
      sr += b[e] * (double)xv.x;
      si += b[e] * (double)xv.y;
    } else {
      sr += b[e] * (double)xv;
    }
  }
  sr = block_sum(sr, sh);
  if (threadIdx.x == 0) coef[(2L * j) * gridDim.x + p] = h3 * sr;
  __syncthreads();
  si = block_sum(si, sh);
  if (threadIdx.x == 0) coef[(2L * j + 1) * gridDim.x + p] = h3 * si;
}

// out_j += E_p c[p][j] beta_p for one projector p (launched per projector: boxes overlap).
template <typename T>
__global__ void k_kb_apply(T* __restrict__ out, int ncols, long Ng, int nx, int ny, int p,
                           int nproj, const int* __restrict__ box,
                           const long long* __restrict__ off, const double* __restrict__ val,
                           const double* __restrict__ Ekb, const double* __restrict__ coef) {
  const int x0 = box[6 * p], y0 = box[6 * p + 1], z0 = box[6 * p + 2];
  const int bx = box[6 * p + 3], by = box[6 * p + 4], bz = box[6 * p + 5];
  const int nb = bx * by * bz, bxy = bx * by;
  const double* b = val + off[p];
  const int j = blockIdx.y;
  const double cr = Ekb[p] * coef[(2L * j) * nproj + p];
  const double ci = Ekb[p] * coef[(2L * j + 1) * nproj + p];
  T* oc = out + (long)j * Ng;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nb; e += gridDim.x * blockDim.x) {
    const int ez = e / bxy, exy = e - ez * bxy, ey = exy / bx, ex = exy - ey * bx;
    const long g = ((long)(z0 + ez) * ny + (y0 + ey)) * nx + x0 + ex;
    if constexpr (sizeof(T) == 2 * sizeof(typename Elem<T>::S)) {
      T o = oc[g];
      o.x += (typename Elem<T>::S)(cr * b[e]);
      o.y += (typename Elem<T>::S)(ci * b[e]);
      oc[g] = o;
    } else {
      oc[g] += (T)(cr * b[e]);
    }
  }
}

template <typename T>
static int apply_h_t(rmgtd_ctx* ctx, const T* x, T* hx, int ncols, const double* vextra) {
  constexpr int BX = 32, BY = 8;
  const int zchunk = 16;
  const int nzc = ceil_div(ctx->nz, zchunk);
  dim3 grid(ceil_div(ctx->nx, BX), ceil_div(ctx->ny, BY), ncols * nzc);
  if ((long)ncols * nzc > 65535L * 1) {
    // blockIdx.z limit: split the columns
    const int per = std::max(1, 65535 / nzc);
    for (int c0 = 0; c0 < ncols; c0 += per) {
      const int nc = std::min(per, ncols - c0);
      int rc = apply_h_t<T>(ctx, x + (long)c0 * ctx->Ng, hx + (long)c0 * ctx->Ng, nc, vextra);
      if (rc) return rc;
    }
    return RMGTD_OK;
  }
  k_hstencil<T, BX, BY><<<grid, dim3(BX, BY), 0, ctx->stream>>>(
      x, hx, ctx->vion, vextra, ctx->nx, ctx->ny, ctx->nz, zchunk, nzc,
      -0.5 / (ctx->h * ctx->h), ctx->Ng);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_hstencil");
  if (ctx->nproj > 0) {
    const int np = ctx->nproj;
    double* coef = kb_coef_buffer(ctx, ncols);
    if (!coef) return set_error(ctx, RMGTD_ENOMEM, "KB coefficient buffer");
    k_kb_project<T><<<dim3(np, ncols), kThreads, 0, ctx->stream>>>(
        x, ncols, ctx->Ng, ctx->nx, ctx->ny, ctx->pbox, ctx->poff, ctx->pval, ctx->h3, coef);
    ++ctx->launches;
    RMGTD_LAUNCH(ctx, "k_kb_project");
    for (int p = 0; p < np; ++p) {
      const long long nb = ctx->h_poff[p + 1] - ctx->h_poff[p];
      if (nb == 0) continue;
      const int bl = (int)std::min<long long>((nb + kThreads - 1) / kThreads, 64);
      k_kb_apply<T><<<dim3(bl, ncols), kThreads, 0, ctx->stream>>>(
          hx, ncols, ctx->Ng, ctx->nx, ctx->ny, p, np, ctx->pbox, ctx->poff, ctx->pval,
          ctx->Ekb, coef);
      ++ctx->launches;
      RMGTD_LAUNCH(ctx, "k_kb_apply");
    }
  }
  return RMGTD_OK;
}

int kb_project_cols(rmgtd_ctx* ctx, const void* x, int ncols, int dtype, double* coef) {
  const int np = ctx->nproj;
  if (np == 0 || ncols == 0) return RMGTD_OK;
  const dim3 grid(np, ncols);
  if (dtype == RMGTD_F64)
    k_kb_project<double><<<grid, kThreads, 0, ctx->stream>>>(
        (const double*)x, ncols, ctx->Ng, ctx->nx, ctx->ny, ctx->pbox, ctx->poff, ctx->pval, ctx->h3, coef);
  else if (dtype == RMGTD_F32)
    k_kb_project<float><<<grid, kThreads, 0, ctx->stream>>>(
        (const float*)x, ncols, ctx->Ng, ctx->nx, ctx->ny, ctx->pbox, ctx->poff, ctx->pval, ctx->h3, coef);
  else
    return set_error(ctx, RMGTD_EINVAL, "kb_project_cols: real columns only");
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_kb_project");
  return RMGTD_OK;
}

int apply_h_dev(rmgtd_ctx* ctx, const void* x, void* hx, int ncols, int dtype,
                const double* vextra) {
  switch (dtype) {
    case RMGTD_F64: return apply_h_t<double>(ctx, (const double*)x, (double*)hx, ncols, vextra);
    case RMGTD_F32: return apply_h_t<float>(ctx, (const float*)x, (float*)hx, ncols, vextra);
    case RMGTD_C128:
      return apply_h_t<double2>(ctx, (const double2*)x, (double2*)hx, ncols, vextra);
    case RMGTD_C64: return apply_h_t<float2>(ctx, (const float2*)x, (float2*)hx, ncols, vextra);
  }
  return set_error(ctx, RMGTD_EINVAL, "unknown dtype");
}


// Mixed-path potential correction of one pass: dv = dV_H + (V_xc(rho0 + drho) - V_xc(rho0)),
// float32 throughout (the float64 fields are rebuilt from the increments when read).  The
// set-up state gives V_ref = V_H,ref + V_xc(rho0) exactly, so no further term enters.
// rho0f: float32 copy of rho0 (NULL: rounded here).
__global__ void k_xc_mixed(const double* __restrict__ rho0, const float* __restrict__ rho0f,
                           const float* __restrict__ drho, const float* __restrict__ dvh,
                           float* __restrict__ dv32, long n, const RepCtl* __restrict__ ctl,
                           long stride, int with_xc, int with_h) {
  const int rep = blockIdx.y;
  if (ctl && !ctl[rep].active) return;
  const long o = rep * stride;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < n;
       g += (long)gridDim.x * blockDim.x) {
    float v = 0.0f;
    if (with_xc) v = dvxc_increment(rho0 + g, rho0f ? rho0f[g] : (float)rho0[g], drho[o + g]);
    if (with_h) v += dvh[o + g];
    dv32[o + g] = v;
  }
}

int launch_xc_mixed(rmgtd_ctx* ctx, const RepCtl* ctl, int nrep) {
  const long n = ctx->Ng;
  const int blocks = (int)std::min<long>(ceil_div(n, kThreads), 4L * ctx->num_sms);
  k_xc_mixed<<<dim3(std::max(blocks, 1), nrep), kThreads, 0, ctx->stream>>>(
      ctx->rho_xc_ref, ctx->rho_ref32, ctx->drho32, ctx->dvh32, ctx->dv32, n, ctl, n,
      ctx->hartree_xc, ctx->hartree_xc);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_xc_mixed");
  return RMGTD_OK;
}

// rho[r][g] = rho_ref[g] + drho[r][g] for every replica (the float64 density of the mixed
// path, rebuilt from its increment; identical to what the density kernels write).
__global__ void k_rho_from_inc(const double* __restrict__ rho_ref, const float* __restrict__ drho,
                               double* __restrict__ rho, long n) {
  const long o = blockIdx.y * n;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < n;
       g += (long)gridDim.x * blockDim.x)
    rho[o + g] = rho_ref[g] + (double)drho[o + g];
}

int rho_from_increment(rmgtd_ctx* ctx) {
  const long n = ctx->Ng;
  const int blocks = (int)std::min<long>(ceil_div(n, kThreads), 4L * ctx->num_sms);
  k_rho_from_inc<<<dim3(std::max(blocks, 1), ctx->nrep), kThreads, 0, ctx->stream>>>(
      ctx->rho_ref, ctx->drho32, ctx->rho, n);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_rho_from_inc");
  return RMGTD_OK;
}

// Stand-alone increment (parity tests): dv[g] = V_xc(rho0[g] + d[g]) - V_xc(rho0[g]).
int launch_xc_increment(rmgtd_ctx* ctx, const double* rho0, const float* d, float* dv, long n) {
  const int blocks = (int)std::min<long>(ceil_div(n, kThreads), 4L * ctx->num_sms);
  k_xc_mixed<<<dim3(std::max(blocks, 1), 1), kThreads, 0, ctx->stream>>>(
      rho0, nullptr, d, nullptr, dv, n, nullptr, n, 1, 0);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_xc_mixed");
  return RMGTD_OK;
}

__global__ void k_lda(const double* __restrict__ rho, double* __restrict__ vh, int vh_mode,
                      const double* __restrict__ vh_ref, float* __restrict__ dvh32,
                      double* __restrict__ vxc, double* __restrict__ exc,
                      double* __restrict__ vhxc, const double* __restrict__ vref,
                      float* __restrict__ dv32, long n, const RepCtl* __restrict__ ctl,
                      long stride, int with_xc, const double* __restrict__ rho_core) {
  const int rep = blockIdx.y;
  if (ctl && !ctl[rep].active) return;
  const long o = rep * stride;
  for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < n;
       g += (long)gridDim.x * blockDim.x) {
    double v = 0.0, e = 0.0;
    if (with_xc) lda_point(rho[o + g] + (rho_core ? rho_core[g] : 0.0), v, e);
    vxc[o + g] = v;
    if (exc) exc[o + g] = e;
    double vhv = 0.0;
    if (vh) {
      if (vh_mode == 1) {
        vhv = vh_ref[g] + (double)dvh32[o + g];
        vh[o + g] = vhv;
      } else {
        vhv = vh[o + g];
        if (vh_mode == 2) dvh32[o + g] = (float)(vhv - vh_ref[g]);
      }
    }
    if (vhxc) vhxc[o + g] = vhv + v;
    if (dv32) dv32[o + g] = (float)(vhv + v - vref[g]);
  }
}

int launch_lda(rmgtd_ctx* ctx, const double* rho, double* vh, int vh_mode, double* vxc,
               double* exc, double* vhxc, float* dv32, long n, const RepCtl* ctl, int nrep,
               long stride, int with_xc, bool with_core) {
  const int blocks = (int)std::min<long>(ceil_div(n, kThreads), 4L * ctx->num_sms);
  k_lda<<<dim3(std::max(blocks, 1), nrep), kThreads, 0, ctx->stream>>>(
      rho, vh, vh_mode, ctx->vh_ref, ctx->dvh32, vxc, exc, vhxc, ctx->vref, dv32, n, ctl, stride,
      with_xc, with_core ? ctx->rho_core : nullptr);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_lda");
  return RMGTD_OK;
}

}  // namespace rmgtd
