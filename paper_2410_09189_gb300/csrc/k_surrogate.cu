// Learned seed of the Hamiltonian self-consistency loop (Algorithm 1's extrapolation).
//
// The paper seeds every step's SCF loop with H_1 = 2 H_0 - H_-1, which is H[V_pred] with
// V_pred = 2 V_0 - V_-1 because H is linear in V.  A small 3-D convolutional network adds a
// correction dV = s_out * y to V_pred, y computed from the last three densities:
//   x[0] = rho_t / s_0,  x[1] = (rho_t - rho_{t-1}) / s_1,  x[2] = (rho_t - 2 rho_{t-1} + rho_{t-2}) / s_2
//   four 3x3x3 cross-correlations, zero padding, 3 -> 16 -> 16 -> 16 -> 1 channels, SiLU after
//   the first three; bfloat16 weights, float32 biases, activations and accumulation.
// The SCF loop still decides convergence, so the converged step does not depend on the
// network; a network with zero last layer is exactly the paper's seed.
//
// Training (on the device, by the kernels below): loss = mean squared error of y against
// the scaled extrapolation residual (V_{t+dt} - 2 V_t + V_{t-dt}) / s_out over the interior
// points (>= 4 from every face) of a batch; gradients by the chain rule (weight gradients
// reduced over blocks in a fixed order, so they do not depend on timing); Adam with
// beta1 = 0.9, beta2 = 0.999, eps = 1e-8 on float32 master parameters, whose bfloat16 copy
// (round to nearest even) the forward pass reads.
//
// Layout: tensors [sample][channel][z][y][x]; parameters per layer W [cout][cin][kz][ky][kx]
// then b [cout] (15,601 floats).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "fastdiv.h"
#include <cstdio>
#include <cstring>

#include "rmgtd_internal.cuh"

namespace rmgtd {
namespace net {

constexpr int kC0 = 3, kC = 16, kLayers = 4;
constexpr int kCin[kLayers] = {3, 16, 16, 16};
constexpr int kCout[kLayers] = {16, 16, 16, 1};
constexpr int kWOff[kLayers] = {0, 1312, 8240, 15168};         // W_l offsets in theta
constexpr int kBOff[kLayers] = {1296, 8224, 15152, 15600};     // b_l offsets
constexpr int kParams = 15601;
constexpr int kRadius = 4;
constexpr float kBeta1 = 0.9f, kBeta2 = 0.999f, kEps = 1e-8f;
constexpr int kFwdThreads = 256;

struct Dims {
  int nx, ny, nz, n;
  FastDiv dx, dy, dn;
};

__device__ __forceinline__ void decode(int g, const Dims& d, int& ix, int& iy, int& iz) {
  const int q = fdiv(g, d.dx);
  ix = g - q * d.nx;
  iz = fdiv(q, d.dy);
  iy = q - iz * d.ny;
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.0f / (1.0f + expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

// ---- forward: one thread per output point, all COUT channels --------------------------------
template <int CIN, int COUT, bool SILU>
__global__ void __launch_bounds__(kFwdThreads)
k_conv_fwd(Dims d, int B, const float* __restrict__ in, const __nv_bfloat16* __restrict__ W,
           const float* __restrict__ bias, float* __restrict__ out, float* __restrict__ pre) {
  __shared__ float Ws[CIN * 27 * COUT];   // [ci][tap][co]
  __shared__ float bs[COUT];
  for (int e = threadIdx.x; e < CIN * 27 * COUT; e += blockDim.x) {
    const int co = e % COUT, r = e / COUT, tap = r % 27, ci = r / 27;
    Ws[e] = __bfloat162float(W[(co * CIN + ci) * 27 + tap]);
  }
  if (threadIdx.x < COUT) bs[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const int plane = d.nx * d.ny;
  const int total = B * d.n;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int b = fdiv(idx, d.dn), g = idx - b * d.n;
    int ix, iy, iz;
    decode(g, d, ix, iy, iz);
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = bs[co];
    for (int ci = 0; ci < CIN; ++ci) {
      const float* src = in + ((long)b * CIN + ci) * d.n + g;
#pragma unroll
      for (int tap = 0; tap < 27; ++tap) {
        const int tz = tap / 9 - 1, ty = (tap / 3) % 3 - 1, tx = tap % 3 - 1;
        const bool ok = (unsigned)(ix + tx) < (unsigned)d.nx && (unsigned)(iy + ty) < (unsigned)d.ny &&
                        (unsigned)(iz + tz) < (unsigned)d.nz;
        const float v = ok ? src[tz * plane + ty * d.nx + tx] : 0.0f;
        const float* w = &Ws[(ci * 27 + tap) * COUT];
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = fmaf(w[co], v, acc[co]);
      }
    }
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
      const long o = ((long)b * COUT + co) * d.n + g;
      if (pre) pre[o] = acc[co];
      out[o] = SILU ? silu(acc[co]) : acc[co];
    }
  }
}

// ---- input gradient of layer l (l >= 1), fused with the SiLU derivative of layer l-1 ---------
// gprev[ci](q) = silu'(z_{l-1}[ci](q)) * sum_co sum_t W[co][ci][t] gz[co](q - t)
template <int CIN, int COUT>
__global__ void __launch_bounds__(kFwdThreads)
k_conv_dgrad(Dims d, int B, const float* __restrict__ gz, const __nv_bfloat16* __restrict__ W,
             const float* __restrict__ zprev, float* __restrict__ gprev) {
  __shared__ float Wt[COUT * 27 * CIN];   // [co][tap][ci]
  for (int e = threadIdx.x; e < COUT * 27 * CIN; e += blockDim.x) {
    const int ci = e % CIN, r = e / CIN, tap = r % 27, co = r / 27;
    Wt[e] = __bfloat162float(W[(co * CIN + ci) * 27 + tap]);
  }
  __syncthreads();
  const int plane = d.nx * d.ny;
  const int total = B * d.n;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int b = fdiv(idx, d.dn), g = idx - b * d.n;
    int ix, iy, iz;
    decode(g, d, ix, iy, iz);
    float acc[CIN];
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.0f;
    for (int co = 0; co < COUT; ++co) {
      const float* src = gz + ((long)b * COUT + co) * d.n + g;
#pragma unroll
      for (int tap = 0; tap < 27; ++tap) {
        const int tz = tap / 9 - 1, ty = (tap / 3) % 3 - 1, tx = tap % 3 - 1;
        // gz at q - t
        const bool ok = (unsigned)(ix - tx) < (unsigned)d.nx && (unsigned)(iy - ty) < (unsigned)d.ny &&
                        (unsigned)(iz - tz) < (unsigned)d.nz;
        const float v = ok ? src[-(tz * plane + ty * d.nx + tx)] : 0.0f;
        const float* w = &Wt[(co * 27 + tap) * CIN];
#pragma unroll
        for (int ci = 0; ci < CIN; ++ci) acc[ci] = fmaf(w[ci], v, acc[ci]);
      }
    }
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
      const long o = ((long)b * CIN + ci) * d.n + g;
      gprev[o] = acc[ci] * silu_grad(zprev[o]);
    }
  }
}

// ---- weight and bias gradients of one layer: per-block partials ------------------------------
// Thread t < CIN*27 owns (ci, tap) and the COUT sums dW[co][ci][tap] over the block's points;
// threads CIN*27 .. CIN*27+COUT-1 own db[co].  The block's points are staged in shared
// memory in chunks of kWgChunk: gz as [p][co], and for every (ci, tap) the input value is
// read through L1.  part[block][kWOff-relative entries..., then biases].
constexpr int kWgChunk = 64;
template <int CIN, int COUT>
__global__ void __launch_bounds__(512)
k_conv_wgrad(Dims d, int B, const float* __restrict__ gz, const float* __restrict__ h,
             float* __restrict__ part) {
  __shared__ float gs[kWgChunk][COUT];
  constexpr int NW = CIN * 27;
  const int t = threadIdx.x;
  const bool wthr = t < NW;
  const bool bthr = !wthr && t < NW + COUT;
  const int ci = wthr ? t / 27 : 0, tap = wthr ? t % 27 : 0;
  const int tz = tap / 9 - 1, ty = (tap / 3) % 3 - 1, tx = tap % 3 - 1;
  const int plane = d.nx * d.ny;
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = 0.0f;
  float bacc = 0.0f;
  const int total = B * d.n;
  const int per = (total + gridDim.x - 1) / gridDim.x;
  const int beg = blockIdx.x * per, end = min(total, beg + per);
  for (int c0 = beg; c0 < end; c0 += kWgChunk) {
    __syncthreads();
    for (int e = t; e < kWgChunk * COUT; e += blockDim.x) {
      const int p = e / COUT, co = e % COUT;
      const int idx = c0 + p;
      float v = 0.0f;
      if (idx < end) {
        const int b = fdiv(idx, d.dn), g = idx - b * d.n;
        v = gz[((long)b * COUT + co) * d.n + g];
      }
      gs[p][co] = v;
    }
    __syncthreads();
    const int np = min(kWgChunk, end - c0);
    if (wthr) {
      for (int p = 0; p < np; ++p) {
        const int idx = c0 + p;
        const int b = fdiv(idx, d.dn), g = idx - b * d.n;
        int ix, iy, iz;
        decode(g, d, ix, iy, iz);
        const bool ok = (unsigned)(ix + tx) < (unsigned)d.nx && (unsigned)(iy + ty) < (unsigned)d.ny &&
                        (unsigned)(iz + tz) < (unsigned)d.nz;
        const float hv = ok ? h[((long)b * CIN + ci) * d.n + g + tz * plane + ty * d.nx + tx] : 0.0f;
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = fmaf(gs[p][co], hv, acc[co]);
      }
    } else if (bthr) {
      const int co = t - NW;
      for (int p = 0; p < np; ++p) bacc += gs[p][co];
    }
  }
  constexpr int P = COUT * CIN * 27 + COUT;
  float* out = part + (long)blockIdx.x * P;
  if (wthr) {
#pragma unroll
    for (int co = 0; co < COUT; ++co) out[(co * CIN + ci) * 27 + tap] = acc[co];
  } else if (bthr) {
    out[COUT * CIN * 27 + (t - NW)] = bacc;
  }
}

// grad[off + e] = sum_blocks part[block][e] (fixed order, float64 accumulation)
__global__ void k_part_reduce(int nblk, int P, const float* __restrict__ part, float* __restrict__ grad) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += (double)part[(long)k * P + e];
    grad[e] = (float)s;
  }
}

// ---- loss: g = 2 m (y - t) / (B n_int); per-block partial sums of m (y - t)^2 ----------------
__global__ void __launch_bounds__(256)
k_loss(Dims d, int B, const float* __restrict__ y, const float* __restrict__ tg, double inv_count,
       float* __restrict__ g, double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  const int total = B * d.n;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int b = fdiv(idx, d.dn), gi = idx - b * d.n;
    int ix, iy, iz;
    decode(gi, d, ix, iy, iz);
    const bool in = ix >= kRadius && ix < d.nx - kRadius && iy >= kRadius && iy < d.ny - kRadius &&
                    iz >= kRadius && iz < d.nz - kRadius;
    const float r = in ? y[idx] - tg[idx] : 0.0f;
    g[idx] = (float)(2.0 * inv_count) * r;
    acc += (double)r * (double)r;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void k_loss_final(int nblk, const double* __restrict__ part, double inv_count,
                             double* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[k];
    *loss = s * inv_count;
  }
}

// ---- Adam on the float32 master parameters; refresh the bfloat16 copy ------------------------
__global__ void k_adam(int P, float* __restrict__ theta, const float* __restrict__ grad,
                       float* __restrict__ m, float* __restrict__ v, float lr, float bc1, float bc2,
                       __nv_bfloat16* __restrict__ wbf) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P; e += gridDim.x * blockDim.x) {
    const float gv = grad[e];
    const float mv = kBeta1 * m[e] + (1.0f - kBeta1) * gv;
    const float vv = kBeta2 * v[e] + (1.0f - kBeta2) * gv * gv;
    m[e] = mv;
    v[e] = vv;
    const float th = theta[e] - lr * (mv / bc1) / (sqrtf(vv / bc2) + kEps);
    theta[e] = th;
    wbf[e] = __float2bfloat16_rn(th);
  }
}

__global__ void k_to_bf16(int P, const float* __restrict__ theta, __nv_bfloat16* __restrict__ wbf) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P; e += gridDim.x * blockDim.x)
    wbf[e] = __float2bfloat16_rn(theta[e]);
}

// ---- features and targets ---------------------------------------------------------------
// x = (rho_t / s0, (rho_t - rho_{t-1}) / s1, (rho_t - 2 rho_{t-1} + rho_{t-2}) / s2); the
// scales arrive as reciprocals (float64 division is slow on this GPU), replica r at r * stride
__global__ void k_features(int n, int nrep, long stride, const double* __restrict__ r0,
                           const double* __restrict__ r1, const double* __restrict__ r2,
                           double i0, double i1, double i2, float* __restrict__ x,
                           double* __restrict__ save) {
  for (int rep = blockIdx.y; rep < nrep; rep += gridDim.y) {
    const double* a0 = r0 + rep * stride;
    const double* a1 = r1 + rep * stride;
    const double* a2 = r2 + rep * stride;
    float* xr = x + (long)rep * 3 * n;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x) {
      const double a = a0[g], b = a1[g], c = a2[g];
      const double d1 = a - b;
      xr[g] = (float)(a * i0);
      xr[n + g] = (float)(d1 * i1);
      xr[2 * n + g] = (float)((d1 - (b - c)) * i2);
      if (save) save[rep * stride + g] = a;
    }
  }
}

__global__ void k_targets(int n, const double* __restrict__ v0, const double* __restrict__ v1,
                          const double* __restrict__ v2, double inv_s, float* __restrict__ t) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < n; g += gridDim.x * blockDim.x)
    t[g] = (float)(((v0[g] - v1[g]) - (v1[g] - v2[g])) * inv_s);
}

// dV = s_out * y into float32 (mixed path) or float64 (float64 path)
__global__ void k_dv_out(long n, const float* __restrict__ y, double s, float* __restrict__ d32,
                         double* __restrict__ d64, const int* __restrict__ failed) {
  if (failed && *failed) return;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const double v = s * (double)y[e];
    if (d32) d32[e] = (float)v;
    if (d64) d64[e] = v;
  }
}

// history after a successful step: h2 <- h1, h1 <- rho at the start of the step
__global__ void k_hist_shift(long n, double* __restrict__ h1, double* __restrict__ h2,
                             const double* __restrict__ start, const int* __restrict__ failed) {
  if (*failed) return;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    h2[e] = h1[e];
    h1[e] = start[e];
  }
}

}  // namespace net
}  // namespace rmgtd

using namespace rmgtd;
using namespace rmgtd::net;

struct rmgtd_net {
  Dims d;
  long Ng = 0;
  int max_batch = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  float* theta = nullptr;            // float32 master parameters
  __nv_bfloat16* wbf = nullptr;      // bfloat16 copy read by the forward pass
  float *m = nullptr, *v = nullptr;  // Adam moments
  float* grad = nullptr;
  int adam_t = 0;
  float* act[kLayers] = {};          // post-activation outputs [B][cout][Ng]
  float* pre[kLayers] = {};          // pre-activations (layers 0..2)
  float* gbuf[2] = {};               // gradient ping-pong [B][16][Ng]
  float* part = nullptr;             // weight-gradient partials
  int part_blocks = 0;
  double* loss_part = nullptr;
  int loss_blocks = 0;
  double* loss_dev = nullptr;
  int* status = nullptr;             // device status word of the tensor-core forward
  double in_scale[3] = {1.0, 1.0, 1.0};
  double out_scale = 1.0;
  std::vector<void*> bufs;
};

namespace {

int net_err(int code, const std::string& msg) { return set_error(nullptr, code, msg); }

#define NET_CUDA(call)                                                                \
  do {                                                                                \
    cudaError_t _e = (call);                                                          \
    if (_e != cudaSuccess) return net_err(RMGTD_ECUDA, std::string(#call ": ") + cudaGetErrorString(_e)); \
  } while (0)
#define NET_LAUNCH(what)                                                              \
  do {                                                                                \
    cudaError_t _e = cudaGetLastError();                                              \
    if (_e != cudaSuccess) return net_err(RMGTD_ECUDA, std::string(what ": ") + cudaGetErrorString(_e)); \
  } while (0)

void* net_alloc(rmgtd_net* n, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) return nullptr;
  n->bufs.push_back(p);
  return p;
}

int grid_for(const rmgtd_net* n, long work, int threads) {
  return (int)std::max<long>(1, std::min<long>((work + threads - 1) / threads, 8L * n->num_sms));
}

}  // namespace

namespace rmgtd {

// forward pass of `batch` samples x [batch][3][Ng] -> y [batch][Ng] on `s`; keep_pre stores
// the pre-activations for a backward pass
int net_forward_on(rmgtd_net* n, const float* x, float* y, int batch, cudaStream_t s, bool keep_pre,
                   bool tc_middle, int* status) {
  const Dims& d = n->d;
  const int gr = grid_for(n, (long)batch * d.n, kFwdThreads);
  const __nv_bfloat16* W = n->wbf;
  const float* th = n->theta;
  k_conv_fwd<3, 16, true><<<gr, kFwdThreads, 0, s>>>(d, batch, x, W + kWOff[0], th + kBOff[0],
                                                      n->act[0], keep_pre ? n->pre[0] : nullptr);
  if (tc_middle && !keep_pre) {
    // the two 16 -> 16 layers on the tensor cores (bfloat16 activations)
    for (int l = 1; l <= 2; ++l) {
      const int rc = conv16_tc(d.nx, d.ny, d.nz, batch, n->act[l - 1], W + kWOff[l], th + kBOff[l],
                               n->act[l], 1, status, n->num_sms, s);
      if (rc) return net_err(rc, "conv16_tc launch failed");
    }
  } else {
    k_conv_fwd<16, 16, true><<<gr, kFwdThreads, 0, s>>>(d, batch, n->act[0], W + kWOff[1],
                                                         th + kBOff[1], n->act[1],
                                                         keep_pre ? n->pre[1] : nullptr);
    k_conv_fwd<16, 16, true><<<gr, kFwdThreads, 0, s>>>(d, batch, n->act[1], W + kWOff[2],
                                                         th + kBOff[2], n->act[2],
                                                         keep_pre ? n->pre[2] : nullptr);
  }
  k_conv_fwd<16, 1, false><<<gr, kFwdThreads, 0, s>>>(d, batch, n->act[2], W + kWOff[3],
                                                       th + kBOff[3], y, nullptr);
  NET_LAUNCH("k_conv_fwd");
  return RMGTD_OK;
}

int net_batch_cap(const rmgtd_net* n) { return n->max_batch; }
long net_grid_points(const rmgtd_net* n, int* nx, int* ny, int* nz) {
  *nx = n->d.nx;
  *ny = n->d.ny;
  *nz = n->d.nz;
  return n->Ng;
}
void net_scales(const rmgtd_net* n, double* s3, double* sout) {
  for (int i = 0; i < 3; ++i) s3[i] = n->in_scale[i];
  *sout = n->out_scale;
}

// ---- context side: predictor at the start of a step, history after it ------------------------
// x from (rho(t), rho(t-dt), rho(t-2dt)) of every replica; y; dV = s_out y; H_1 += h^3 Phi^T dV Phi
int net_predict(rmgtd_ctx* ctx) {
  rmgtd_net* n = ctx->net;
  const long Ng = ctx->Ng;
  const int nrep = ctx->nrep;
  const int bl = (int)std::max<long>(1, std::min<long>(ceil_div(Ng * nrep, 256L), 8L * ctx->num_sms));
  k_features<<<dim3(std::max(1, bl / nrep), nrep), 256, 0, ctx->stream>>>(
      (int)Ng, nrep, Ng, ctx->rho, ctx->rho_h1, ctx->rho_h2, 1.0 / n->in_scale[0],
      1.0 / n->in_scale[1], 1.0 / n->in_scale[2], ctx->net_x, ctx->rho_start);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_features");
  int rc = net_forward_on(n, ctx->net_x, ctx->net_y, nrep, ctx->stream, false, true, ctx->status);
  if (rc) return set_error(ctx, rc, rmgtd_last_error(nullptr));
  ctx->launches += kLayers;
  k_dv_out<<<bl, 256, 0, ctx->stream>>>(Ng * nrep, ctx->net_y, n->out_scale,
                                        ctx->mixed ? ctx->net_dv32 : nullptr,
                                        ctx->mixed ? nullptr : ctx->net_dv64, ctx->failed);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_dv_out");
  // H_1[r] += h^3 Phi^T diag(dV_r) Phi: the base is each replica's own H_1
  const long NN = (long)ctx->N * ctx->N;
  if (ctx->mixed)
    return gram_mixed(ctx, ctx->net_dv32, Ng, nrep, ctx->h3, ctx->H1, ctx->H1, ctx->ctl, nullptr, NN);
  return gram(ctx, ctx->phi, ctx->phi, ctx->net_dv64, Ng, nrep, ctx->h3, ctx->H1, ctx->H1, nullptr,
              ctx->ctl, 1, nullptr, NN);
}

int net_history_shift(rmgtd_ctx* ctx) {
  const long n = ctx->Ng * ctx->nrep;
  const int bl = (int)std::max<long>(1, std::min<long>(ceil_div(n, 256L), 8L * ctx->num_sms));
  k_hist_shift<<<bl, 256, 0, ctx->stream>>>(n, ctx->rho_h1, ctx->rho_h2, ctx->rho_start, ctx->failed);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_hist_shift");
  return RMGTD_OK;
}

// no history (creation, kick, load, set_matrix, attach): rho(t-dt) = rho(t-2dt) = rho(t)
int net_history_reset(rmgtd_ctx* ctx) {
  if (!ctx->rho_h1) return RMGTD_OK;
  const size_t bytes = sizeof(double) * ctx->Ng * ctx->nrep;
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->rho_h1, ctx->rho, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->rho_h2, ctx->rho, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  return RMGTD_OK;
}

}  // namespace rmgtd

// ---- C ABI ----------------------------------------------------------------------------------
extern "C" {

long long rmgtd_net_num_params(void) { return kParams; }

int rmgtd_net_create(int nx, int ny, int nz, int max_batch, void* stream, rmgtd_net** out) {
  if (!out) return net_err(RMGTD_EINVAL, "net_create: out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1 || max_batch < 1)
    return net_err(RMGTD_EINVAL, "net_create: empty grid or batch");
  const long long Ng = (long long)nx * ny * nz;
  if (Ng * max_batch * kC >= (1ll << 31))
    return net_err(RMGTD_EINVAL, "net_create: batch * 16 * grid points must be below 2^31");
  rmgtd_net* n = new rmgtd_net();
  n->d.nx = nx;
  n->d.ny = ny;
  n->d.nz = nz;
  n->d.n = (int)Ng;
  n->d.dx = make_fastdiv(nx);
  n->d.dy = make_fastdiv(ny);
  n->d.dn = make_fastdiv((int)Ng);
  n->Ng = Ng;
  n->max_batch = max_batch;
  n->stream = (cudaStream_t)stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (n->num_sms < 1) n->num_sms = 1;
  const size_t act = sizeof(float) * (size_t)max_batch * kC * Ng;
  bool ok = true;
  auto A = [&](size_t b) {
    void* p = net_alloc(n, b);
    ok = ok && p;
    return p;
  };
  n->theta = (float*)A(sizeof(float) * kParams);
  n->wbf = (__nv_bfloat16*)A(sizeof(__nv_bfloat16) * kParams);
  n->m = (float*)A(sizeof(float) * kParams);
  n->v = (float*)A(sizeof(float) * kParams);
  n->grad = (float*)A(sizeof(float) * kParams);
  for (int l = 0; l < kLayers - 1; ++l) {
    n->act[l] = (float*)A(act);
    n->pre[l] = (float*)A(act);
  }
  n->gbuf[0] = (float*)A(act);
  n->gbuf[1] = (float*)A(act);
  n->part_blocks = 2 * n->num_sms;
  n->part = (float*)A(sizeof(float) * (size_t)n->part_blocks * (16 * 16 * 27 + 16));
  n->loss_blocks = 2 * n->num_sms;
  n->loss_part = (double*)A(sizeof(double) * n->loss_blocks);
  n->loss_dev = (double*)A(sizeof(double));
  n->status = (int*)A(sizeof(int));
  if (!ok) {
    rmgtd_net_destroy(n);
    return net_err(RMGTD_ENOMEM, "net_create: device memory");
  }
  cudaMemsetAsync(n->theta, 0, sizeof(float) * kParams, n->stream);
  cudaMemsetAsync(n->wbf, 0, sizeof(__nv_bfloat16) * kParams, n->stream);
  cudaMemsetAsync(n->m, 0, sizeof(float) * kParams, n->stream);
  cudaMemsetAsync(n->v, 0, sizeof(float) * kParams, n->stream);
  if (cudaStreamSynchronize(n->stream) != cudaSuccess) {
    rmgtd_net_destroy(n);
    return net_err(RMGTD_ECUDA, "net_create: initialisation");
  }
  *out = n;
  return RMGTD_OK;
}

void rmgtd_net_destroy(rmgtd_net* n) {
  if (!n) return;
  if (n->stream) cudaStreamSynchronize(n->stream);
  for (void* p : n->bufs) cudaFree(p);
  delete n;
}

int rmgtd_net_set_params(rmgtd_net* n, const float* theta_host) {
  if (!n || !theta_host) return net_err(RMGTD_EINVAL, "net_set_params: NULL argument");
  NET_CUDA(cudaMemcpyAsync(n->theta, theta_host, sizeof(float) * kParams, cudaMemcpyHostToDevice, n->stream));
  k_to_bf16<<<grid_for(n, kParams, 256), 256, 0, n->stream>>>(kParams, n->theta, n->wbf);
  NET_LAUNCH("k_to_bf16");
  NET_CUDA(cudaMemsetAsync(n->m, 0, sizeof(float) * kParams, n->stream));
  NET_CUDA(cudaMemsetAsync(n->v, 0, sizeof(float) * kParams, n->stream));
  n->adam_t = 0;
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return RMGTD_OK;
}

int rmgtd_net_get_params(rmgtd_net* n, float* theta_host) {
  if (!n || !theta_host) return net_err(RMGTD_EINVAL, "net_get_params: NULL argument");
  NET_CUDA(cudaMemcpyAsync(theta_host, n->theta, sizeof(float) * kParams, cudaMemcpyDeviceToHost, n->stream));
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return RMGTD_OK;
}

int rmgtd_net_set_scales(rmgtd_net* n, const double in_scales[3], double out_scale) {
  if (!n || !in_scales) return net_err(RMGTD_EINVAL, "net_set_scales: NULL argument");
  for (int i = 0; i < 3; ++i)
    if (!(in_scales[i] > 0) || !isfinite(in_scales[i]))
      return net_err(RMGTD_EINVAL, "net_set_scales: scales must be positive and finite");
  if (!(out_scale > 0) || !isfinite(out_scale))
    return net_err(RMGTD_EINVAL, "net_set_scales: scales must be positive and finite");
  for (int i = 0; i < 3; ++i) n->in_scale[i] = in_scales[i];
  n->out_scale = out_scale;
  return RMGTD_OK;
}

int rmgtd_net_get_scales(rmgtd_net* n, double in_scales[3], double* out_scale) {
  if (!n || !in_scales || !out_scale) return net_err(RMGTD_EINVAL, "net_get_scales: NULL argument");
  for (int i = 0; i < 3; ++i) in_scales[i] = n->in_scale[i];
  *out_scale = n->out_scale;
  return RMGTD_OK;
}

int rmgtd_net_features(rmgtd_net* n, const double* rho_t, const double* rho_tm1,
                       const double* rho_tm2, float* x_dev) {
  if (!n || !rho_t || !rho_tm1 || !rho_tm2 || !x_dev)
    return net_err(RMGTD_EINVAL, "net_features: NULL argument");
  k_features<<<grid_for(n, n->Ng, 256), 256, 0, n->stream>>>(
      (int)n->Ng, 1, n->Ng, rho_t, rho_tm1, rho_tm2, 1.0 / n->in_scale[0], 1.0 / n->in_scale[1],
      1.0 / n->in_scale[2], x_dev, nullptr);
  NET_LAUNCH("k_features");
  return RMGTD_OK;
}

int rmgtd_net_targets(rmgtd_net* n, const double* v_tp1, const double* v_t, const double* v_tm1,
                      float* t_dev) {
  if (!n || !v_tp1 || !v_t || !v_tm1 || !t_dev) return net_err(RMGTD_EINVAL, "net_targets: NULL argument");
  k_targets<<<grid_for(n, n->Ng, 256), 256, 0, n->stream>>>((int)n->Ng, v_tp1, v_t, v_tm1,
                                                            1.0 / n->out_scale, t_dev);
  NET_LAUNCH("k_targets");
  return RMGTD_OK;
}

int rmgtd_net_forward(rmgtd_net* n, const float* x_dev, float* y_dev, int batch) {
  if (!n || !x_dev || !y_dev) return net_err(RMGTD_EINVAL, "net_forward: NULL argument");
  if (batch < 1 || batch > n->max_batch) return net_err(RMGTD_EINVAL, "net_forward: batch out of range");
  int rc = net_forward_on(n, x_dev, y_dev, batch, n->stream, false, false, n->status);
  if (rc) return rc;
  NET_CUDA(cudaStreamSynchronize(n->stream));
  return RMGTD_OK;
}

int rmgtd_net_forward_tc(rmgtd_net* n, const float* x_dev, float* y_dev, int batch) {
  if (!n || !x_dev || !y_dev) return net_err(RMGTD_EINVAL, "net_forward_tc: NULL argument");
  if (batch < 1 || batch > n->max_batch) return net_err(RMGTD_EINVAL, "net_forward_tc: batch out of range");
  NET_CUDA(cudaMemsetAsync(n->status, 0, sizeof(int), n->stream));
  int rc = net_forward_on(n, x_dev, y_dev, batch, n->stream, false, true, n->status);
  if (rc) return rc;
  int st = 0;
  NET_CUDA(cudaMemcpyAsync(&st, n->status, sizeof(int), cudaMemcpyDeviceToHost, n->stream));
  NET_CUDA(cudaStreamSynchronize(n->stream));
  if (st) return net_err(st, "net_forward_tc: device wait timed out");
  return RMGTD_OK;
}

int rmgtd_net_backward(rmgtd_net* n, const float* x_dev, const float* t_dev, int batch,
                       double* loss, float* grad_host) {
  if (!n || !x_dev || !t_dev) return net_err(RMGTD_EINVAL, "net_backward: NULL argument");
  if (batch < 1 || batch > n->max_batch) return net_err(RMGTD_EINVAL, "net_backward: batch out of range");
  const Dims& d = n->d;
  const int nin = std::max(0, d.nx - 2 * kRadius) * std::max(0, d.ny - 2 * kRadius) *
                  std::max(0, d.nz - 2 * kRadius);
  if (nin == 0) return net_err(RMGTD_EINVAL, "net_backward: grid has no interior points");
  const double inv_count = 1.0 / ((double)batch * nin);
  cudaStream_t s = n->stream;
  // forward with the pre-activations; the output goes to gbuf[1] (reused below)
  float* y = n->gbuf[1];
  int rc = net_forward_on(n, x_dev, y, batch, s, true, false, n->status);
  if (rc) return rc;
  float* g = n->gbuf[0];
  k_loss<<<n->loss_blocks, 256, 0, s>>>(d, batch, y, t_dev, inv_count, g, n->loss_part);
  k_loss_final<<<1, 32, 0, s>>>(n->loss_blocks, n->loss_part, inv_count, n->loss_dev);
  NET_LAUNCH("k_loss");
  const int gr = grid_for(n, (long)batch * d.n, kFwdThreads);
  const int pb = n->part_blocks;
  // layer 3 (16 -> 1, no activation): weight gradient, then the input gradient with SiLU'
  k_conv_wgrad<16, 1><<<pb, 512, 0, s>>>(d, batch, g, n->act[2], n->part);
  k_part_reduce<<<32, 256, 0, s>>>(pb, 16 * 27 + 1, n->part, n->grad + kWOff[3]);
  k_conv_dgrad<16, 1><<<gr, kFwdThreads, 0, s>>>(d, batch, g, n->wbf + kWOff[3], n->pre[2], n->gbuf[1]);
  NET_LAUNCH("layer 3 backward");
  // layer 2
  k_conv_wgrad<16, 16><<<pb, 512, 0, s>>>(d, batch, n->gbuf[1], n->act[1], n->part);
  k_part_reduce<<<32, 256, 0, s>>>(pb, 16 * 16 * 27 + 16, n->part, n->grad + kWOff[2]);
  k_conv_dgrad<16, 16><<<gr, kFwdThreads, 0, s>>>(d, batch, n->gbuf[1], n->wbf + kWOff[2], n->pre[1], n->gbuf[0]);
  NET_LAUNCH("layer 2 backward");
  // layer 1
  k_conv_wgrad<16, 16><<<pb, 512, 0, s>>>(d, batch, n->gbuf[0], n->act[0], n->part);
  k_part_reduce<<<32, 256, 0, s>>>(pb, 16 * 16 * 27 + 16, n->part, n->grad + kWOff[1]);
  k_conv_dgrad<16, 16><<<gr, kFwdThreads, 0, s>>>(d, batch, n->gbuf[0], n->wbf + kWOff[1], n->pre[0], n->gbuf[1]);
  NET_LAUNCH("layer 1 backward");
  // layer 0 (input gradient not needed)
  k_conv_wgrad<3, 16><<<pb, 512, 0, s>>>(d, batch, n->gbuf[1], x_dev, n->part);
  k_part_reduce<<<32, 256, 0, s>>>(pb, 16 * 3 * 27 + 16, n->part, n->grad + kWOff[0]);
  NET_LAUNCH("layer 0 backward");
  if (loss) NET_CUDA(cudaMemcpyAsync(loss, n->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
  if (grad_host)
    NET_CUDA(cudaMemcpyAsync(grad_host, n->grad, sizeof(float) * kParams, cudaMemcpyDeviceToHost, s));
  NET_CUDA(cudaStreamSynchronize(s));
  return RMGTD_OK;
}

int rmgtd_net_adam(rmgtd_net* n, double lr) {
  if (!n) return net_err(RMGTD_EINVAL, "net_adam: NULL net");
  if (!(lr > 0) || !isfinite(lr)) return net_err(RMGTD_EINVAL, "net_adam: lr must be positive");
  n->adam_t += 1;
  const float bc1 = (float)(1.0 - pow((double)kBeta1, n->adam_t));
  const float bc2 = (float)(1.0 - pow((double)kBeta2, n->adam_t));
  k_adam<<<grid_for(n, kParams, 256), 256, 0, n->stream>>>(kParams, n->theta, n->grad, n->m, n->v,
                                                          (float)lr, bc1, bc2, n->wbf);
  NET_LAUNCH("k_adam");
  return RMGTD_OK;
}

// Weight file: 8-byte tag "RMGTDNET", uint32 version 1, uint32 reserved 0, int64 parameter
// count, float64 feature scales s_0..s_2 and output scale, then the float32 parameters; all
// little-endian as written by the host.
static const char kNetTag[8] = {'R', 'M', 'G', 'T', 'D', 'N', 'E', 'T'};

int rmgtd_net_save(rmgtd_net* n, const char* path) {
  if (!n || !path) return net_err(RMGTD_EINVAL, "net_save: NULL argument");
  std::vector<float> theta(kParams);
  int rc = rmgtd_net_get_params(n, theta.data());
  if (rc) return rc;
  FILE* fp = fopen(path, "wb");
  if (!fp) return net_err(RMGTD_EINVAL, std::string("net_save: cannot open ") + path);
  const uint32_t ver = 1, res = 0;
  const int64_t count = kParams;
  const double sc[4] = {n->in_scale[0], n->in_scale[1], n->in_scale[2], n->out_scale};
  bool ok = fwrite(kNetTag, 1, 8, fp) == 8 && fwrite(&ver, 4, 1, fp) == 1 &&
            fwrite(&res, 4, 1, fp) == 1 && fwrite(&count, 8, 1, fp) == 1 &&
            fwrite(sc, 8, 4, fp) == 4 &&
            fwrite(theta.data(), sizeof(float), kParams, fp) == (size_t)kParams;
  ok = (fclose(fp) == 0) && ok;
  return ok ? RMGTD_OK : net_err(RMGTD_EINVAL, std::string("net_save: write failed: ") + path);
}

int rmgtd_net_load(rmgtd_net* n, const char* path) {
  if (!n || !path) return net_err(RMGTD_EINVAL, "net_load: NULL argument");
  FILE* fp = fopen(path, "rb");
  if (!fp) return net_err(RMGTD_EINVAL, std::string("net_load: cannot open ") + path);
  char tag[8];
  uint32_t ver = 0, res = 0;
  int64_t count = 0;
  double sc[4];
  std::vector<float> theta(kParams);
  bool ok = fread(tag, 1, 8, fp) == 8 && memcmp(tag, kNetTag, 8) == 0 && fread(&ver, 4, 1, fp) == 1 &&
            ver == 1 && fread(&res, 4, 1, fp) == 1 && fread(&count, 8, 1, fp) == 1 &&
            count == kParams && fread(sc, 8, 4, fp) == 4 &&
            fread(theta.data(), sizeof(float), kParams, fp) == (size_t)kParams;
  char extra;
  ok = ok && fread(&extra, 1, 1, fp) == 0;   // nothing after the parameters
  fclose(fp);
  if (!ok) return net_err(RMGTD_EINVAL, std::string("net_load: not a weight file of this network: ") + path);
  for (float t : theta)
    if (!isfinite(t)) return net_err(RMGTD_EINVAL, "net_load: non-finite parameter");
  int rc = rmgtd_net_set_scales(n, sc, sc[3]);
  if (rc) return rc;
  return rmgtd_net_set_params(n, theta.data());
}

}  // extern "C"
