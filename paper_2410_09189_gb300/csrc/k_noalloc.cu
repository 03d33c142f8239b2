// Allocation-free Gram contraction: C = scale * A^T diag(w) B for orbital blocks already in
// device memory, with its split-over-the-grid scratch in a fixed device array of this file
// instead of memory from cudaMalloc or an allocator hook.
//
// Who needs it: callers that must not allocate device memory at the point of the call --
// code running while a stream is being captured into a CUDA graph (cudaMalloc is not
// permitted there), hosts that own every byte of device memory through their own arena and
// forbid library allocations, and latency-critical loops that cannot afford the implicit
// synchronisation of cudaMalloc/cudaFree.  The context-based API (rmgtd_create) allocates
// its buffers up front and is unsuitable for them.
//
// The scratch array is shared by every call in the process on a given GPU and keeps the
// last call's contents: calls whose work overlaps on the device race on it.  Each call
// overwrites every scratch element it later reads, so nothing needs clearing.
#include <cuda.h>   // CUcontext (the driver entry point comes from the runtime)

#include <mutex>

#include "rmgtd_internal.cuh"

namespace {

constexpr long long kScratchDoubles = 1ll << 20;  // 8 MiB of float64 partial sums
constexpr int kTile = 32;
constexpr int kMaxSplit = 64;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_gram_scratch[kScratchDoubles];

// device address of g_gram_scratch per device ordinal, with the CUDA context it was looked
// up in: a different current context on that device (after cudaDeviceReset, or a primary
// context torn down and rebuilt) makes the next call look the address up again
double* g_scratch_addr[kMaxDevices] = {nullptr};
CUcontext g_scratch_ctx[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// cuCtxGetCurrent through the runtime's driver entry point (no link to libcuda); NULL when
// unavailable, in which case the address is looked up on every call
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<CtxGetCurrentFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// partial[split][i*N + j] = sum over the split's grid range of A[i][g] w[g] B[j][g]
__global__ void __launch_bounds__(256)
k_gram_split_static(int N, long long Ng, const double* __restrict__ A,
                    const double* __restrict__ B, const double* __restrict__ w, long long chunk,
                    double* __restrict__ part) {
  __shared__ double As[kTile][kTile + 1];
  __shared__ double Bs[kTile][kTile + 1];
  const int T = (N + kTile - 1) / kTile;
  const int I = blockIdx.x / T, J = blockIdx.x % T;
  const int split = blockIdx.y;
  const long long g_beg = (long long)split * chunk;
  const long long g_end = min(Ng, g_beg + chunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc00 = 0, acc01 = 0, acc10 = 0, acc11 = 0;
  for (long long g0 = g_beg; g0 < g_end; g0 += kTile) {
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + 256 * e;
      const int r = idx >> 5, c = idx & 31;
      const long long g = g0 + c;
      const int ia = I * kTile + r, jb = J * kTile + r;
      double av = 0.0, bv = 0.0;
      if (g < g_end) {
        if (ia < N) av = A[(long long)ia * Ng + g];
        if (jb < N) {
          bv = B[(long long)jb * Ng + g];
          if (w) bv *= w[g];
        }
      }
      As[c][r] = av;
      Bs[c][r] = bv;
    }
    __syncthreads();
    for (int k = 0; k < kTile; ++k) {
      const double a0 = As[k][ty], a1 = As[k][ty + 16];
      const double b0 = Bs[k][tx], b1 = Bs[k][tx + 16];
      acc00 = fma(a0, b0, acc00);
      acc01 = fma(a0, b1, acc01);
      acc10 = fma(a1, b0, acc10);
      acc11 = fma(a1, b1, acc11);
    }
    __syncthreads();
  }
  double* out = part + (long long)split * N * N;
  const int i0 = I * kTile + ty, i1 = i0 + 16, j0 = J * kTile + tx, j1 = j0 + 16;
  if (i0 < N && j0 < N) out[(long long)i0 * N + j0] = acc00;
  if (i0 < N && j1 < N) out[(long long)i0 * N + j1] = acc01;
  if (i1 < N && j0 < N) out[(long long)i1 * N + j0] = acc10;
  if (i1 < N && j1 < N) out[(long long)i1 * N + j1] = acc11;
}

// C[e] = scale * sum_split partial[split][e], summed in split order
__global__ void k_gram_sum_static(int N, int nsplit, const double* __restrict__ part,
                                  double scale, double* __restrict__ C) {
  const long long NN = (long long)N * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NN;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < nsplit; ++k) s += part[(long long)k * NN + e];
    C[e] = scale * s;
  }
}

}  // namespace

extern "C" int rmgtd_gram_noalloc(const double* a_dev, const double* b_dev, const double* w_dev,
                                  int n_orb, long long n_grid, double scale, double* c_dev,
                                  void* stream) {
  using rmgtd::set_error;
  if (!a_dev || !b_dev || !c_dev || n_orb < 1 || n_grid < 1)
    return set_error(nullptr, RMGTD_EINVAL, "gram_noalloc: NULL pointer or empty size");
  const long long NN = (long long)n_orb * n_orb;
  if (NN > kScratchDoubles)
    return set_error(nullptr, RMGTD_EINVAL,
                     "gram_noalloc: n_orb^2 exceeds the fixed scratch of 1048576 doubles "
                     "(n_orb <= 1024)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(nullptr, RMGTD_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(nullptr, RMGTD_EINVAL, "gram_noalloc: device ordinal out of range");
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    CUcontext cur = nullptr;
    const CtxGetCurrentFn get = ctx_get_current();
    const bool known = get && get(&cur) == CUDA_SUCCESS && cur;
    if (!g_scratch_addr[dev] || !known || g_scratch_ctx[dev] != cur) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_gram_scratch);
      if (e != cudaSuccess)
        return set_error(nullptr, RMGTD_ECUDA,
                         std::string("gram_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = (double*)p;
      g_scratch_ctx[dev] = known ? cur : nullptr;
    }
    scratch = g_scratch_addr[dev];
  }
  long long ns = kScratchDoubles / NN;
  if (ns > kMaxSplit) ns = kMaxSplit;
  const long long by_grid = (n_grid + 255) / 256;
  if (ns > by_grid) ns = by_grid;
  if (ns < 1) ns = 1;
  const int nsplit = (int)ns;
  const long long chunk = ((n_grid + nsplit - 1) / nsplit + kTile - 1) / kTile * kTile;
  const int T = (n_orb + kTile - 1) / kTile;
  cudaStream_t s = (cudaStream_t)stream;
  k_gram_split_static<<<dim3(T * T, nsplit), 256, 0, s>>>(n_orb, n_grid, a_dev, b_dev, w_dev,
                                                           chunk, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(nullptr, RMGTD_ECUDA, cudaGetErrorString(e));
  const int bl = (int)((NN + 255) / 256 < 1024 ? (NN + 255) / 256 : 1024);
  k_gram_sum_static<<<bl, 256, 0, s>>>(n_orb, nsplit, scratch, scale, c_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(nullptr, RMGTD_ECUDA, cudaGetErrorString(e));
  return RMGTD_OK;
}
