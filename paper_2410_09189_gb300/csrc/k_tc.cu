// Tensor-core (tcgen05) kernels of the mixed path.
//
// Density change (Algorithm 1's rho(P_1), Section 3.1's rho = sum_ij Re P_ij phi_i phi_j)
// as a GEMM on the 5th-generation tensor cores:
//   Y_r(g, j) = sum_k phi_k(g) Shat_r[k][j]        (M = 128 grid points, N = 32 nrep, K = 32)
//   drho_r(g) = sum_j phi_j(g) Y_r(g, j)            (epilogue, one thread per grid point)
// with Shat_r the float32 upper-triangular change matrix (2 (S - S_ref)_kj for k < j,
// (S - S_ref)_jj on the diagonal).  Operands are float32 split as x = hi + lo with hi = x
// rounded down to tf32 (low 13 mantissa bits cleared) and lo = x - hi (exact); the three
// products hi*hi + hi*lo + lo*hi accumulate in float32 in tensor memory (kind::tf32), which
// keeps about 2^-20 relative accuracy (the dropped lo*lo term and the tf32 truncation of lo).
//
// Shared-memory operands use the canonical K-major layout without swizzle: core matrices
// of 8 rows x 16 bytes (4 floats), the K-adjacent core matrix at +128 bytes (leading byte
// offset), the next group of 8 rows at +K/4 * 128 bytes (stride byte offset).  The density
// kernel (k_rho_ws) is persistent and warp-specialised: per 128-point tile one bulk copy of
// the tiled orbitals, four converter warps building the operands, one issuer warp issuing the
// MMAs into one of two tensor-memory accumulators, and the converters forming drho of the
// previous tile while the tensor cores work on the current one.
#include <string.h>

#include <algorithm>

#include "tc_common.cuh"

namespace rmgtd {
namespace tc {

constexpr int kM = 128;          // grid points per tile = TMEM lanes
constexpr int kK = 32;           // orbitals per tile (N <= 32)
constexpr int kMaxRepTc = 8;     // N = 32 * nrep <= 256
constexpr uint32_t kSBO = (kK / 4) * 128;             // 1024 B between 8-row groups
constexpr uint32_t kLBO = 128;                        // K-adjacent core matrices


// float index of element (row, k) in a K-major no-swizzle tile with K = kK
__device__ __forceinline__ int kmaj(int row, int k) {
  return (row >> 3) * (kSBO / 4) + (k >> 2) * (kLBO / 4) + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((kSBO >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::tf32, D float32, A and B tf32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}





// Density, warp-specialised and persistent (one CTA per SM, 128-point tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ...): an issuer warp keeps kRhoStages tiles of the 32-point-tiled
// orbitals in flight (one 16 KB cp.async.bulk per tile: 4 contiguous 4 KB blocks) and issues
// each tile's 12 MMAs; nt teams of four warps (thread <-> point) take the tiles in turn
// (tile i -> team i % nt, with its own K-major operand buffer and tensor-memory accumulator):
// a team converts its tile (hi/lo split) and then, while the tensor cores work on it, forms
// drho of its previous tile from its accumulator.  mbarriers between the roles: full[s]
// (loads -> teams), afull[b] (operands written, load slot free -> issuer), mdone[b] (MMAs
// done -> team), tfree[b] (accumulator read -> issuer).  All waits bounded; a time-out
// aborts every role and drains the loads.
constexpr int kRhoStages = 4;
constexpr int kRhoMaxTeams = 3;
constexpr int kRhoTileB = kM * kK * 4;        // 16 KB of tiled orbitals per tile
constexpr int kMomRep = 4;                    // replicas whose moments the kernel forms




// dynamic shared memory: raw[kRhoStages][128 x 32], A[nt] (hi, lo: 128 x 32 each), B (hi, lo:
// nr * 32 x 32 each); blockDim = 32 (4 nt + 1)
__global__ void __launch_bounds__(32 * (4 * kRhoMaxTeams + 1), 1)
k_rho_ws(int N, int Np, int Ng, int nr, int nt, const float* __restrict__ phit,
         const float* __restrict__ shat, const double* __restrict__ rho_ref,
         double* __restrict__ rho, float* __restrict__ drho, const RepCtl* __restrict__ ctl,
         int* status, double* __restrict__ mom, int nx, int ny, int nz, float hgrid) {
  extern __shared__ __align__(128) float sm[];
  __shared__ __align__(8) uint64_t full[kRhoStages];
  __shared__ __align__(8) uint64_t afull[kRhoMaxTeams], mdone[kRhoMaxTeams], tfree[kRhoMaxTeams];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int committed;                         // tiles whose MMAs were committed
  __shared__ float momw[4 * kRhoMaxTeams][4 * kMomRep];     // per-warp moment sums
  float* raw = sm;                                  // kRhoStages x 4096 floats
  float* abuf = sm + kRhoStages * kM * kK;          // nt x (hi, lo)
  float* b_hi = abuf + nt * 2 * kM * kK;
  float* b_lo = b_hi + nr * 32 * kK;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ncols_used = nr * 32;
  uint32_t acc_cols = 32;
  while (acc_cols < (uint32_t)ncols_used) acc_cols <<= 1;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)nt * acc_cols) ncols <<= 1;   // nt accumulators
  const int ntiles = (Ng + kM - 1) / kM;
  const int ntl = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  volatile int* abort_v = &abort_flag;
  const int issuer_warp = 4 * nt;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    abort_flag = 0;
    committed = 0;
    for (int s = 0; s < kRhoStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[s])) : "memory");
    for (int b = 0; b < nt; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(saddr(&afull[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mdone[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(saddr(&tfree[b])) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // B operand once: row n = r * 32 + j, column k: Shat_r[k][j] (zero beyond N)
  for (int e = tid; e < ncols_used * kK; e += blockDim.x) {
    const int k = e / ncols_used, n = e - k * ncols_used;
    const int r = n >> 5, j = n & 31;
    float v = 0.0f;
    if (j < N && k < N) v = shat[((long)r * Np + k) * Np + j];
    float hi, lo;
    split_tf32(v, hi, lo);
    b_hi[kmaj(n, k)] = hi;
    b_lo[kmaj(n, k)] = lo;
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == issuer_warp) {
    // ---- issuer warp -------------------------------------------------------------------
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(kM, ncols_used);
      auto issue = [&](int i) {
        const int t = blockIdx.x + i * gridDim.x;
        const int s = i % kRhoStages;
        const uint32_t bar = saddr(&full[s]);
        mbar_expect_tx(bar, (uint32_t)kRhoTileB);
        bulk_g2s_1d(saddr(raw + s * kM * kK), phit + (long)t * kM * kK, (uint32_t)kRhoTileB, bar);
      };
      int issued = 0;
      for (; issued < min(kRhoStages, ntl); ++issued) issue(issued);
      for (int i = 0; i < ntl; ++i) {
        const int b = i % nt;
        bool ok = mbar_wait(&afull[b], (uint32_t)(i / nt) & 1u);
        if (ok && i + kRhoStages < ntl) {   // the team is done with slot i % kRhoStages
          issue(i + kRhoStages);
          issued = i + kRhoStages + 1;
        }
        if (ok && i >= nt) ok = mbar_wait(&tfree[b], (uint32_t)((i - nt) / nt) & 1u);
        if (!ok || *abort_v) {
          *abort_v = 1;
          break;
        }
        fence_after();
        const float* a = abuf + b * 2 * kM * kK;
        const uint32_t ah = saddr(a), al = saddr(a + kM * kK), bh = saddr(b_hi), bl = saddr(b_lo);
        const uint32_t d = tbase + (uint32_t)(b * acc_cols);
#pragma unroll
        for (int s = 0; s < kK / 8; ++s) {
          const uint32_t off = s * 2 * kLBO;
          mma_tf32(d, sdesc(ah + off), sdesc(bh + off), idesc, s > 0 ? 1u : 0u);
          mma_tf32(d, sdesc(ah + off), sdesc(bl + off), idesc, 1u);
          mma_tf32(d, sdesc(al + off), sdesc(bh + off), idesc, 1u);
        }
        mma_commit(&mdone[b]);
        *reinterpret_cast<volatile int*>(&committed) = i + 1;
      }
      // loads still in flight after an abort: wait for every issued stage (bounded)
      if (*abort_v)
        for (int u = max(0, issued - kRhoStages); u < issued; ++u)
          mbar_wait(&full[u % kRhoStages], (uint32_t)(u / kRhoStages) & 1u);
    }
    __syncwarp();
  } else if (warp < issuer_warp) {
    // ---- team warps: team = warp / 4, thread <-> point p = tid % 128 of the tile ------------
    const int team = warp >> 2;
    const int p = tid & (kM - 1);
    const int wq = warp & 3;                        // TMEM lane quadrant of this warp
    float ph[kK], pv[kK];   // this tile's and the team's previous tile's values at p
    unsigned on_mask = 0;   // replicas to write (active ones)
    for (int r = 0; r < nr; ++r)
      if (!ctl || ctl[r].active) on_mask |= 1u << r;
    // multipole moments of drho (charge, dipole about the box centre) for the Hartree
    // solve's boundary values, summed per thread over its points
    float mq[kMomRep][4];
#pragma unroll
    for (int r = 0; r < kMomRep; ++r) mq[r][0] = mq[r][1] = mq[r][2] = mq[r][3] = 0.0f;
    const float cx = 0.5f * (float)(nx - 1), cy = 0.5f * (float)(ny - 1), cz = 0.5f * (float)(nz - 1);
    auto epilogue = [&](int i) {   // drho of tile i from accumulator i % nt
      const int b = i % nt;
      if (!mbar_wait(&mdone[b], (uint32_t)(i / nt) & 1u)) {
        *abort_v = 1;
        return false;
      }
      fence_after();
      const int g = (blockIdx.x + i * gridDim.x) * kM + p;
      float xq = 0.0f, yq = 0.0f, zq = 0.0f;
      if (mom && g < Ng) {
        const int ix = g % nx, rest = g / nx;
        xq = ((float)ix - cx) * hgrid;
        yq = ((float)(rest % ny) - cy) * hgrid;
        zq = ((float)(rest / ny) - cz) * hgrid;
      }
      for (int r = 0; r < nr; ++r) {
        float y[32];
        tmem_ld32(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(b * acc_cols + r * 32), y);
        float acc = 0.0f;
#pragma unroll
        for (int j = 0; j < 32; ++j) acc = fmaf(pv[j], y[j], acc);
        if (g < Ng && ((on_mask >> r) & 1u)) {
          if (rho) rho[(long)r * Ng + g] = rho_ref[g] + (double)acc;
          drho[(long)r * Ng + g] = acc;
#pragma unroll
          for (int rr = 0; rr < kMomRep; ++rr)   // register-indexed (r is not a constant)
            if (rr == r) {
              mq[rr][0] += acc;
              mq[rr][1] += acc * xq;
              mq[rr][2] += acc * yq;
              mq[rr][3] += acc * zq;
            }
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[b]);
      return true;
    };
    int prev = -1;
    for (int i = team; i < ntl; i += nt) {
      const int s = i % kRhoStages, b = i % nt;
      bool ok = mbar_wait(&full[s], (uint32_t)(i / kRhoStages) & 1u);
      if (ok && i >= nt) ok = mbar_wait(&mdone[b], (uint32_t)((i - nt) / nt) & 1u);  // A[b] free
      if (!ok || *abort_v) {
        *abort_v = 1;
        break;
      }
      // this point's 32 orbital values: 32-point block p / 32, row k, column p % 32
      const float* rs = raw + s * kM * kK + (p >> 5) * (kK * 32) + (p & 31);
#pragma unroll
      for (int k = 0; k < kK; ++k) ph[k] = rs[k * 32];
      float* a_hi = abuf + b * 2 * kM * kK;
      float* a_lo = a_hi + kM * kK;
#pragma unroll
      for (int kc = 0; kc < kK; kc += 4) {
        float4 h4, l4;
        split_tf32(ph[kc], h4.x, l4.x);
        split_tf32(ph[kc + 1], h4.y, l4.y);
        split_tf32(ph[kc + 2], h4.z, l4.z);
        split_tf32(ph[kc + 3], h4.w, l4.w);
        *reinterpret_cast<float4*>(&a_hi[kmaj(p, kc)]) = h4;
        *reinterpret_cast<float4*>(&a_lo[kmaj(p, kc)]) = l4;
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&afull[b]);
      // while the tensor cores work on tile i: drho of this team's previous tile
      if (prev >= 0 && !epilogue(prev)) break;
#pragma unroll
      for (int k = 0; k < kK; ++k) pv[k] = ph[k];
      prev = i;
    }
    if (!*abort_v && prev >= 0) epilogue(prev);
    if (mom) {   // warp sums of the moments, one row of momw per team warp
#pragma unroll
      for (int r = 0; r < kMomRep; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float v = warp_sumf(mq[r][q]);
          if (lane == 0 && r < nr) momw[warp][r * 4 + q] = v;
        }
    }
  }
  __syncthreads();
  // block moments: fixed order over the team warps, float64, one partial per CTA
  if (mom && tid < 4 * nr) {
    double sacc = 0.0;
    for (int w = 0; w < 4 * nt; ++w) sacc += (double)momw[w][tid];
    mom[(long)tid * gridDim.x + blockIdx.x] = sacc;
  }
  if (*abort_v && tid == 0) atomicCAS(status, 0, (int)RMGTD_ETIMEOUT);
  // every committed MMA has completed before the accumulators are freed: each team waited on
  // its tiles' mdone; after an abort wait for the last committed one (its commit covers the
  // earlier ones; bounded)
  if (*abort_v && tid == 0) {
    const int c = *reinterpret_cast<volatile int*>(&committed);
    if (c > 0) mbar_wait(&mdone[(c - 1) % nt], (uint32_t)((c - 1) / nt) & 1u);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols)
                 : "memory");
  }
}

}  // namespace tc

// Density of the mixed path on the tensor cores (N <= 32, nrep <= 8); returns 1 when the
// shape is outside that range (the caller then uses the float32 SIMT kernel).
int rho_tc(rmgtd_ctx* ctx, double* rho, float* drho, const RepCtl* ctl, int nrep) {
  using namespace tc;
  const int N = ctx->N, Np = ((N + 31) / 32) * 32;
  if (Np != kK || nrep > kMaxRepTc || ctx->Ng >= (1l << 31)) return 1;
  // teams: three while three accumulators fit the 512 tensor-memory columns, else two
  const int acc = nrep <= 1 ? 32 : nrep <= 2 ? 64 : nrep <= 4 ? 128 : 256;
  const int nt = (3 * acc <= 512) ? 3 : 2;
  const size_t smem =
      (size_t)(kRhoStages * kM * kK + nt * 2 * kM * kK + 2 * nrep * 32 * kK) * sizeof(float);
  if (!ctx->rho_tc_attr) {   // the largest layout (3 teams, kMaxRepTc replicas), set once
    RMGTD_CUDA(ctx, cudaFuncSetAttribute(
                        k_rho_ws, cudaFuncAttributeMaxDynamicSharedMemorySize,
                        (int)((kRhoStages * kM * kK + 3 * 2 * kM * kK + 2 * kMaxRepTc * 32 * kK) * 4)));
    ctx->rho_tc_attr = 1;
  }
  const int ntiles = (int)((ctx->Ng + kM - 1) / kM);
  const int grid = std::min(ntiles, ctx->num_sms);
  // multipole moments of drho for the Hartree solve that follows (partials per CTA)
  double* mom = nullptr;
  if (ctx->rho_mom && nrep <= kMomRep && (long)4 * nrep * grid <= ctx->rho_mom_cap)
    mom = ctx->rho_mom;
  k_rho_ws<<<grid, 32 * (4 * nt + 1), smem, ctx->stream>>>(
      N, Np, (int)ctx->Ng, nrep, nt, ctx->phi32t, ctx->shat32, ctx->rho_ref, rho, drho, ctl,
      ctx->status, mom, ctx->nx, ctx->ny, ctx->nz, (float)ctx->h);
  ctx->rho_mom_blocks = mom ? grid : 0;
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_rho_ws");
  return RMGTD_OK;
}

namespace tc {

// ---- float32 Gram partials on the tensor cores ---------------------------------------------
// H update of the mixed path (Algorithm 1's density-functional update, Section 3.1's H = h^3 Phi^T (V Phi)):
//   G_r[i][j] = sum_g (w_r(g) phi_i(g)) phi_j(g)     for the orbital tile pair (It, Jt)
// as D = A B^T with M = 128 rows (4 replicas x 32 orbitals of tile It, w-weighted), N = 32
// (orbitals of tile Jt), K = grid points, accumulated in tensor memory over the CTA's chunk
// of the grid (split-K; k_gram32_reduce adds the chunks in a fixed order).  3xTF32 as in
// k_rho_ws.  Warp-specialised pipeline over 32-point stages: an issuer warp (one elected
// thread) keeps a ring of S stages of tiled TMA loads in flight (cp.async.bulk.tensor.2d,
// completion on an mbarrier per slot) -- the 32 x 32 orbital box of tile It (and Jt) and the
// 4 x 32 weight box -- and issues the 12 MMAs of each converted stage, committing to that
// operand buffer's mbarrier; eight converter warps turn each stage into one of nb operand
// buffers (weight product, hi/lo split, K-major core-matrix layout) and arrive on its
// mbarrier.  No block-wide barrier inside the loop: the roles wait on each other's
// mbarriers only (bounded; a time-out aborts every role and drains the loads).  The boxes use
// the 128-byte swizzle (16-byte chunk c of row r stored at chunk c ^ (r mod 8)), so the
// conversion's 16-byte shared loads of 8 rows are conflict-free; its stores write whole
// 128-byte core-matrix rows per quarter warp.  Rows past N, points past Ng and replicas past
// nrep arrive as zeros (the tensor maps' out-of-bounds fill).
constexpr int kGKS = 32;                        // grid points per stage (K)
constexpr int kGAfl = 128 * kGKS;               // floats per A operand (hi or lo)
constexpr int kGBfl = 32 * kGKS;                // floats per B operand (hi or lo)
constexpr int kGOpF = 2 * kGAfl + 2 * kGBfl;    // one operand buffer (40 KB)
constexpr int kThreadsConv = 256;             // converter warps
constexpr int kThreadsG = kThreadsConv + 32;    // + one TMA / MMA issuer warp
constexpr int kGMaxStages = 16;
constexpr int kGMaxOpBufs = 3;

constexpr int kGBoxB = 32 * kGKS * 4;           // bytes of one 32 x 32 orbital box
constexpr int kGWBoxB = 4 * kGKS * 4;           // bytes of the 4 x 32 weight box

// raw slot: orbital box It [, box Jt], weight box; 1024-byte multiples (swizzle atoms)
__host__ __device__ constexpr int gram_slot_bytes(bool two_tiles) {
  return (two_tiles ? 2 : 1) * kGBoxB + 1024;
}


// 4 floats at row r, column 4 q of a 128-byte-swizzled box of 32-float rows
__device__ __forceinline__ float4 swz_ld4(const float* box, int r, int q) {
  return *reinterpret_cast<const float4*>(box + r * 32 + ((q ^ (r & 7)) << 2));
}


__global__ void __launch_bounds__(kThreadsG, 1)
k_gram_tc(const __grid_constant__ CUtensorMap tm_phi, const __grid_constant__ CUtensorMap tm_w,
          int N, int Np, int Ng, int nrep, int T, int chunk, int S, int nb,
          float* __restrict__ part, const RepCtl* __restrict__ ctl, int* status) {
  extern __shared__ __align__(128) float sm[];
  __shared__ __align__(8) uint64_t full[kGMaxStages];   // TMA -> converters
  __shared__ __align__(8) uint64_t conv[kGMaxOpBufs];   // converters -> issuer
  __shared__ __align__(8) uint64_t mdone[kGMaxOpBufs];  // MMAs -> converters
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ int issued_n;                              // stages whose loads were issued
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int It, Jt;
  {
    int i = 0, rem = blockIdx.y;
    while (rem >= T - i) {
      rem -= T - i;
      ++i;
    }
    It = i;
    Jt = i + rem;
  }
  const bool diag = (It == Jt);
  const bool two = T > 1;                       // slot layout of this launch
  const int slotB = gram_slot_bytes(two);
  const int wbox = (two ? 2 : 1) * kGBoxB;      // weight box within a slot (bytes)
  const int rep0 = blockIdx.z * 4;
  const int nr = min(4, nrep - rep0);
  const int g_beg = blockIdx.x * chunk;
  const int g_end = min(Ng, g_beg + chunk);
  const int nst = g_end > g_beg ? (g_end - g_beg + kGKS - 1) / kGKS : 0;
  float* op = sm;                               // nb operand buffers
  // S raw slots from the first 1024-byte boundary after the operands (swizzle atoms)
  const uint32_t raw_s = (saddr(sm + nb * kGOpF) + 1023u) & ~1023u;
  const float* raw = sm + (raw_s - saddr(sm)) / 4;
  const uint32_t ncols = 32;
  constexpr int kConvWarps = kThreadsConv / 32;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    abort_flag = 0;
    issued_n = 0;
    for (int s = 0; s < S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&full[s])) : "memory");
    for (int b = 0; b < nb; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(&conv[b])),
                   "r"(kConvWarps)
                   : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mdone[b])) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // operand rows of replicas >= nr stay zero
  for (int e = tid; e < nb * kGOpF; e += blockDim.x) op[e] = 0.0f;
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = tmem_base;
  volatile int* abort_v = &abort_flag;
  volatile int* issued_v = &issued_n;

  if (warp == kConvWarps) {
    // ---- issuer warp: TMA loads into the ring, MMAs of converted stages ------------------
    // Each box arrives whole (out-of-bounds elements zero-filled), so the transaction count
    // is fixed; x = g0 is a multiple of 32.
    auto issue = [&](int t) {
      const int slot = t % S;
      const int g0 = g_beg + t * kGKS;
      const uint32_t bar = saddr(&full[slot]);
      const uint32_t base = raw_s + (uint32_t)(slot * slotB);
      mbar_expect_tx(bar, (uint32_t)((diag ? 1 : 2) * kGBoxB + kGWBoxB));
        // tiled orbitals: the 32 x 32 block (point tile g0/32, orbital tile) is contiguous
      const int row0 = (g0 >> 5) * Np;
      tma_load_2d(base, &tm_phi, 0, row0 + It * 32, bar);
      if (!diag) tma_load_2d(base + kGBoxB, &tm_phi, 0, row0 + Jt * 32, bar);
      tma_load_2d(base + wbox, &tm_w, g0, rep0, bar);
      *issued_v = t + 1;
    };
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(128, 32);
      for (int u = 0; u < min(S, nst); ++u) issue(u);
      for (int t = 0; t < nst; ++t) {
        const int ob = t % nb;
        if (!mbar_wait(&conv[ob], (uint32_t)(t / nb) & 1u) || *abort_v) {
          *abort_v = 1;
          break;
        }
        fence_after();
        const float* o = op + ob * kGOpF;
        const uint32_t sah = saddr(o), sal = saddr(o + kGAfl), sbh = saddr(o + 2 * kGAfl),
                       sbl = saddr(o + 2 * kGAfl + kGBfl);
#pragma unroll
        for (int k = 0; k < kGKS / 8; ++k) {
          const uint32_t off = k * 2 * kLBO;
          mma_tf32(tbase, sdesc(sah + off), sdesc(sbh + off), idesc, (t > 0 || k > 0) ? 1u : 0u);
          mma_tf32(tbase, sdesc(sah + off), sdesc(sbl + off), idesc, 1u);
          mma_tf32(tbase, sdesc(sal + off), sdesc(sbh + off), idesc, 1u);
        }
        mma_commit(&mdone[ob]);
        // the converters are done with raw slot t % S: refill it with stage t + S
        if (t + S < nst) issue(t + S);
      }
    }
    __syncwarp();
  } else {
    // ---- converter warps: raw boxes -> operand buffers ------------------------------------
    // a quarter warp covers 8 consecutive rows at one 4-point column
    const int i = 8 * (warp & 3) + (lane & 7);
    const int q = (lane >> 3) + 4 * (warp >> 2);
    for (int t = 0; t < nst; ++t) {
      const int slot = t % S, ob = t % nb;
      bool ok = mbar_wait(&full[slot], (uint32_t)(t / S) & 1u);
      if (ok && t >= nb) ok = mbar_wait(&mdone[ob], (uint32_t)((t - nb) / nb) & 1u);
      if (!ok || *abort_v) {
        *abort_v = 1;
        break;
      }
      fence_after();
      const float* rs = raw + slot * (slotB / 4);
      // points past the chunk end (inside the grid: the next CTA's) are masked here
      const int nv = min(kGKS, g_end - (g_beg + t * kGKS));
      const bool in = 4 * q < nv;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      if (in) a = swz_ld4(rs, i, q);
      if (diag)
        b = a;
      else if (in)
        b = swz_ld4(rs + kGBoxB / 4, i, q);
      float* o = op + ob * kGOpF;
      float* ah = o;
      float* al = o + kGAfl;
      float* bh = o + 2 * kGAfl;
      float* bl = o + 2 * kGAfl + kGBfl;
      for (int r = 0; r < nr; ++r) {
        float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (in) wv = swz_ld4(rs + wbox / 4, r, q);
        float4 h4, l4;
        split_tf32(a.x * wv.x, h4.x, l4.x);
        split_tf32(a.y * wv.y, h4.y, l4.y);
        split_tf32(a.z * wv.z, h4.z, l4.z);
        split_tf32(a.w * wv.w, h4.w, l4.w);
        *reinterpret_cast<float4*>(&ah[kmaj(r * 32 + i, 4 * q)]) = h4;
        *reinterpret_cast<float4*>(&al[kmaj(r * 32 + i, 4 * q)]) = l4;
      }
      {
        float4 h4, l4;
        split_tf32(b.x, h4.x, l4.x);
        split_tf32(b.y, h4.y, l4.y);
        split_tf32(b.z, h4.z, l4.z);
        split_tf32(b.w, h4.w, l4.w);
        *reinterpret_cast<float4*>(&bh[kmaj(i, 4 * q)]) = h4;
        *reinterpret_cast<float4*>(&bl[kmaj(i, 4 * q)]) = l4;
      }
      // operands visible to the tensor cores, raw slot released: one arrival per warp
      fence_async_smem();
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(&conv[ob]))
                     : "memory");
    }
  }
  __syncthreads();
  // drain: the last MMAs (their commit covers all earlier ones) and, after an abort, the TMA
  // loads still in flight into this CTA's shared memory (every issued stage completes)
  bool ok = !*abort_v;
  if (tid == 0) {
    bool drained = true;
    if (nst > 0 && ok)
      drained = mbar_wait(&mdone[(nst - 1) % nb], (uint32_t)((nst - 1) / nb) & 1u);
    if (!ok) {
      // wait for the last issued stage of every slot (phases complete in order; a completed
      // phase returns at once), so no load is still writing when the CTA exits
      const int n_iss = *issued_v;
      for (int u = max(0, n_iss - S); u < n_iss; ++u) mbar_wait(&full[u % S], (uint32_t)(u / S) & 1u);
      drained = false;
    }
    if (!drained) {
      atomicCAS(status, 0, (int)RMGTD_ETIMEOUT);
      *abort_v = 1;
    }
  }
  __syncthreads();
  ok = !*abort_v;
  fence_after();
  // epilogue: TMEM lane m = 32 warp + lane is A row (replica rep0 + warp, orbital It*32+lane)
  if (ok && warp < nr) {
    float y[32];
    if (nst > 0) {
      tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16), y);
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) y[j] = 0.0f;
    }
    const int r = rep0 + warp;
    const bool on = !ctl || ctl[r].active;
    const long NpNp = (long)Np * Np;
    float* out = part + ((long)blockIdx.x * nrep + r) * NpNp + (long)(It * 32 + lane) * Np + Jt * 32;
    // diagonal tile pairs: only j >= i is read by the reduction (4-column groups from the
    // one holding the diagonal)
    const int j0 = diag ? (lane & ~3) : 0;
#pragma unroll
    for (int j = 0; j < 32; j += 4)
      if (j >= j0)
        *reinterpret_cast<float4*>(out + j) =
            on ? make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols)
                 : "memory");
  }
}

}  // namespace tc

// float32 Gram partials on the tensor cores; returns 1 when the shapes are outside its
// range (the caller then runs the SIMT kernel), else the status.  Partials as k_gram32.
namespace {


// rows x Ng float32 matrix with row stride Ng (a multiple of 4): boxes of 32 points x
// box_rows rows, 128-byte swizzle, zero fill out of bounds
bool encode_rows(void* map, const float* base, long Ng, int rows, int box_rows) {
  const EncodeTiledFn f = tensor_map_encoder();
  if (!f) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)Ng, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Ng * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)tc::kGKS, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  return f(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
           const_cast<float*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

// float32 Gram partials on the tensor cores; returns 1 when the shapes are outside its
// range or the tensor maps cannot be made (the caller then runs the SIMT kernel), else the
// status.  Partials as k_gram32.
int gram_tc(rmgtd_ctx* ctx, const float* w, int nw, float* part, int nsplit, int chunk,
            const RepCtl* ctl) {
  using namespace tc;
  static_assert(sizeof(CUtensorMap) == sizeof(ctx->tm_phi), "tensor map size");
  const int N = ctx->N;
  const int T = ceil_div(N, 32);
  const int Np = T * 32;
  // tensor maps want 16-byte row strides; boxes start at multiples of 32 points
  if (ctx->Ng >= (1l << 31) || ctx->Ng % 4 || chunk % kGKS ||
      ceil_div(ctx->Ng, 32L) * Np >= (1l << 31))
    return 1;
  if (!ctx->tm_phi_ok) {
    if (!encode_rows(ctx->tm_phi, ctx->phi32t, 32, (int)(ceil_div(ctx->Ng, 32L) * Np), 32))
      return 1;
    ctx->tm_phi_ok = 1;
  }
  if (ctx->tm_w_key != (const void*)w || ctx->tm_w_rows != nw) {
    if (!encode_rows(ctx->tm_w, w, ctx->Ng, nw, 4)) return 1;
    ctx->tm_w_key = w;
    ctx->tm_w_rows = nw;
  }
  const int per_sm = std::max(1, std::min(ctx->tune_gram_blocks, 2));
  const size_t budget = (per_sm == 1 ? 220 : 110) * 1024;
  const int nb = per_sm == 1 ? 3 : 2;                        // operand buffers
  const size_t slot = gram_slot_bytes(T > 1);
  const size_t fixed = sizeof(float) * nb * kGOpF + 1024;   // operands + swizzle alignment
  const int S = (int)std::min<size_t>(kGMaxStages, (budget - fixed) / slot);
  if (S < 2) return 1;
  const size_t smem = fixed + S * slot;
  // the attribute belongs to the function (process-wide): only ever raise it
  if (ctx->gram_tc_attr < (int)smem) {
    cudaFuncAttributes fa;
    RMGTD_CUDA(ctx, cudaFuncGetAttributes(&fa, k_gram_tc));
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
      RMGTD_CUDA(ctx, cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
    ctx->gram_tc_attr = (int)smem;
  }
  CUtensorMap tm_phi, tm_w;
  memcpy(&tm_phi, ctx->tm_phi, sizeof(tm_phi));
  memcpy(&tm_w, ctx->tm_w, sizeof(tm_w));
  const dim3 grid(nsplit, T * (T + 1) / 2, ceil_div(nw, 4));
  k_gram_tc<<<grid, kThreadsG, smem, ctx->stream>>>(tm_phi, tm_w, N, Np, (int)ctx->Ng, nw, T,
                                                      chunk, S, nb, part, ctl, ctx->status);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gram_tc");
  return RMGTD_OK;
}

// ---- 16 -> 16 channel 3x3x3 convolution of the learned seed on the tensor cores -------------
// Inference form of the network's two middle layers (the propagation's predictor): implicit
// GEMM with M = 128 output points, N = 16 output channels, K = 16 input channels per tap,
// one kind::f16 MMA per tap (27 taps accumulate in tensor memory).  Activations are rounded
// to bfloat16 when staged (the weights already are); accumulation is float32.  A tile of 128
// consecutive points (flat index over samples and points) is staged as K-major operands
// A_t[p][c] = x_c(p + t) (zero outside the grid), one 16-byte store per 8 channels, nine
// taps (one z offset) at a time: the 72 loads of a group are in flight together, and the
// 51 KB of shared memory let four CTAs share an SM.
namespace tc {

constexpr int kCvM = 128;                  // points per tile
constexpr int kCvC = 16;                   // channels in and out
constexpr int kCvThreads = 256;
constexpr int kCvAbytes = kCvM * kCvC * 2; // one tap's A operand (4 KB)
constexpr int kCvBbytes = kCvC * kCvC * 2; // one tap's B operand (512 B)

// bf16 index of element (row, k) in a K-major no-swizzle operand with K = 16: core matrices
// of 8 rows x 8 bf16, K-adjacent at +128 B, 8-row groups at +256 B
__device__ __forceinline__ int kmaj16(int row, int k) {
  return (row >> 3) * 128 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}


__device__ __forceinline__ uint64_t sdesc_lbo_sbo(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}




__global__ void __launch_bounds__(kCvThreads)
k_conv16_tc(int nx, int ny, int nz, int B, const float* __restrict__ in,
            const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
            float* __restrict__ out, int silu, int* status) {
  extern __shared__ __align__(128) unsigned char smc[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ float bs[kCvC];
  // A: one group of 9 taps (a z offset) at a time; B: all 27 taps
  __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(smc);
  __nv_bfloat16* Bw = reinterpret_cast<__nv_bfloat16*>(smc + 9 * kCvAbytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = nx * ny * nz, plane = nx * ny;
  const int total = B * n;
  const uint32_t ncols = 32;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&tmem_base)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < kCvC) bs[tid] = bias[tid];
  // B_t[co][ci] = W[co][ci][t]
  for (int e = tid; e < 27 * kCvC * kCvC; e += blockDim.x) {
    const int t = e / (kCvC * kCvC), r = e % (kCvC * kCvC), co = r / kCvC, ci = r % kCvC;
    Bw[t * (kCvBbytes / 2) + kmaj16(co, ci)] = W[(co * kCvC + ci) * 27 + t];
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = idesc_bf16(kCvM, kCvC);
  const int ntiles = (total + kCvM - 1) / kCvM;
  const int p = tid & (kCvM - 1), half = tid >> 7;   // point of the tile, channels 8 half ..
  uint32_t phase = 0;
  bool ok_all = true;
  for (int tile = blockIdx.x; tile < ntiles && ok_all; tile += gridDim.x) {
    const int idx = tile * kCvM + p;
    const bool valid = idx < total;
    int b = 0, g = 0, ix = 0, iy = 0, iz = 0;
    if (valid) {
      b = idx / n;
      g = idx - b * n;
      ix = g % nx;
      const int q = g / nx;
      iy = q % ny;
      iz = q / ny;
    }
    const float* src = in + ((long)b * kCvC + 8 * half) * n;
    for (int grp = 0; grp < 3; ++grp) {   // taps with z offset grp - 1
      const int tz = grp - 1;
      const bool zok = valid && (unsigned)(iz + tz) < (unsigned)nz;
      float v[9][8];
#pragma unroll
      for (int u = 0; u < 9; ++u) {       // all 72 loads of the group in flight together
        const int ty = u / 3 - 1, tx = u % 3 - 1;
        const bool ok = zok && (unsigned)(ix + tx) < (unsigned)nx && (unsigned)(iy + ty) < (unsigned)ny;
        const int off = g + tz * plane + ty * nx + tx;
#pragma unroll
        for (int c = 0; c < 8; ++c) v[u][c] = ok ? src[(long)c * n + off] : 0.0f;
      }
      if (grp > 0) {   // the MMAs of the previous group read A
        const bool okw = mbar_wait(&bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!okw)) {
          ok_all = false;
          break;
        }
        fence_after();
      }
#pragma unroll
      for (int u = 0; u < 9; ++u) {
        uint4 w4;
        w4.x = pack_bf16(v[u][0], v[u][1]);
        w4.y = pack_bf16(v[u][2], v[u][3]);
        w4.z = pack_bf16(v[u][4], v[u][5]);
        w4.w = pack_bf16(v[u][6], v[u][7]);
        *reinterpret_cast<uint4*>(&A[u * (kCvAbytes / 2) + kmaj16(p, 8 * half)]) = w4;
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        fence_after();
        const uint32_t a0 = saddr(A), b0 = saddr(Bw);
        for (int u = 0; u < 9; ++u) {
          const int t = 9 * grp + u;
          mma_bf16(tbase, sdesc_lbo_sbo(a0 + u * kCvAbytes, 128, 256),
                   sdesc_lbo_sbo(b0 + t * kCvBbytes, 128, 256), idesc, t > 0 ? 1u : 0u);
        }
        mma_commit(&bar);
      }
    }
    if (!ok_all) break;
    const bool okw = mbar_wait(&bar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!okw)) {
      ok_all = false;
      break;
    }
    fence_after();
    if (warp < 4) {   // TMEM lanes 32 warp .. : points of the tile
      float y[16];
      tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16), y);
      const int pi = tile * kCvM + warp * 32 + lane;
      if (pi < total) {
        const int bb = pi / n, gg = pi - bb * n;
#pragma unroll
        for (int co = 0; co < kCvC; ++co) {
          const float z = y[co] + bs[co];
          out[((long)bb * kCvC + co) * n + gg] = silu ? z / (1.0f + expf(-z)) : z;
        }
      }
    }
    fence_before();
    __syncthreads();
  }
  if (!ok_all && tid == 0) atomicCAS(status, 0, (int)RMGTD_ETIMEOUT);
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols)
                 : "memory");
  }
}

}  // namespace tc

// y = conv(x) (+ SiLU) for a 16 -> 16 layer on the tensor cores, on stream s.
int conv16_tc(int nx, int ny, int nz, int B, const float* x, const __nv_bfloat16* W,
              const float* bias, float* y, int silu, int* status, int num_sms, cudaStream_t s) {
  using namespace tc;
  static bool attr = false;
  const size_t smem = 9 * (size_t)kCvAbytes + 27 * (size_t)kCvBbytes;
  if (!attr) {
    if (cudaFuncSetAttribute(k_conv16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
      return RMGTD_ECUDA;
    attr = true;
  }
  const long total = (long)B * nx * ny * nz;
  const int ntiles = (int)((total + kCvM - 1) / kCvM);
  const int grid = std::min(ntiles, 4 * num_sms);   // 4 CTAs (51 KB each) per SM
  k_conv16_tc<<<grid, kCvThreads, smem, s>>>(nx, ny, nz, B, x, W, bias, y, silu, status);
  return cudaGetLastError() == cudaSuccess ? RMGTD_OK : RMGTD_ECUDA;
}

}  // namespace rmgtd
