// Orbital-tiled tensor-core contractions of the mixed path for active spaces of 32 < N <= 256
// orbitals (Section 3.1: rho = sum_ij Re P_ij phi_i phi_j and H = h^3 Phi^T V Phi; Table 1's
// "Rho" and "Hupdate", the two largest phases of a step).
//
// Operands: the orbitals are stored once, at set-up, as two bfloat16 planes Phi = hi + lo
// (hi = Phi rounded to bfloat16, lo = the rest rounded again; |Phi - hi - lo| <= 2^-17 |Phi|),
// in 64-point blocks [2][nblk][Np][64] (Np = N rounded up to 32, nblk = Ng / 64 rounded up,
// zeros beyond): every operand box of a TMA copy -- 64 points of 64 orbitals for the density,
// 64 points of all Np orbitals for the Gram -- is one contiguous run of memory, so the copies
// read whole DRAM pages instead of 128-byte pieces of rows Ng values apart.  Every product a*b is formed on the tensor cores as a_hi b_hi + a_hi b_lo + a_lo b_hi
// (kind::f16, bfloat16 inputs, float32 accumulation in tensor memory): about 2^-16 relative
// per product, with the same four bytes per orbital value as a float32 copy.  All operand
// tiles arrive by TMA with the 128-byte swizzle; no per-replica padding.
//
// Anchors: both contractions work on the change since the replica's anchor, a consistent
// pair of states moved to the new state after every completed step (rho(Sa) with Sa, and
// Ha = H(Va) with Va): drho = drho_a + sum (S - Sa)_ij phi_i phi_j and
// H = Ha + h^3 Phi^T diag(V - Va) Phi.  The split's rounding then scales with one step's
// change, so the SCF loop converges as on the float64 path; the float64 reference state of
// the set-up (rho_ref, V_ref) stays the origin of drho and dV.
//
// Density change (k_rho_planes), per replica r and 128-point tile:
//   D[g][j] = sum_{k <= j} phi_k(g) Shat_r[k][j]    (M = 128 points, N = Np - 64 c, K = orbitals)
//   drho_r(g) = sum_j phi_j(g) D[g][j]
// Shat_r is upper triangular (2 dS_kj for k < j, dS_jj on the diagonal, dS = Re P - Sa_r), so
// the K loop runs over 64-orbital chunks c and chunk c only adds to columns j >= 64 c: after
// chunk c's MMAs, columns [64 c, 64 c + 64) are final, and the epilogue forms their part of
// drho from the same shared-memory chunk (the orbitals are read from HBM once) while the
// tensor cores go on with chunk c + 1.  Shat's planes stay in shared memory for the launch.
//
// Gram (k_gram_planes), per replica r and grid chunk (split-K):
//   G_r[i][j] = sum_g (w_r(g) phi_i(g)) phi_j(g)   (M = 128 orbitals i, N = Np - 128 I, K = points)
// One TMA copy per 64-point stage brings all Np orbital rows (both planes); converter warps
// form the weighted A operands w * (hi + lo) -> bfloat16 hi / lo for the row tiles I = 0, 1
// (same swizzled positions); only the upper block triangle is multiplied.  Partials
// [split][replica][Np][Np] go to k_gram32_reduce (fixed-order sum, float64 result, SCF error).
#include <string.h>

#include <algorithm>

#include "tc_common.cuh"

namespace rmgtd {
namespace tc {

constexpr int kPK = 64;                  // bf16 elements per 128-byte row (stage / chunk width)
constexpr int kPM = 128;                 // MMA M = TMEM lanes
constexpr int kPMaxNp = 256;
constexpr int kPlaneBox = kPK * kPK * 2; // one 64 x 64 bf16 box (8 KB)
constexpr int kRdSlotB = 4 * kPlaneBox;  // density chunk: hi box0, hi box1, lo box0, lo box1
constexpr int kRdMaxSlots = 4;
constexpr int kRdThreads = 6 * 32;       // TMA producer, MMA issuer, 4 epilogue warps
constexpr int kGConvWarps = 16;          // converter / epilogue warps of the Gram
constexpr int kGpThreads = (2 + kGConvWarps) * 32;   // + TMA producer and MMA issuer
constexpr int kGpMaxStages = 6;   // raw slots of the Gram's copy ring
constexpr int kSmemLimit = 226 * 1024;   // dynamic part (static barriers take the rest)

__device__ __forceinline__ uint4 lds_u4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a));
  return v;
}
__device__ __forceinline__ float lds_f(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_u4(uint32_t a, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}

__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }

// x -> (hi, lo) bfloat16 pair, round to nearest even; packs two points per 32-bit word
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& h, uint32_t& l) {
  const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(hb);
  const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  h = *reinterpret_cast<const uint32_t*>(&hb);
  l = *reinterpret_cast<const uint32_t*>(&lb);
}

// ---- set-up and per-pass operand preparation ------------------------------------------------
// planes[0][b][k][q] = hi, planes[1][b][k][q] = lo of phi_k(64 b + q) (zero past N and Ng)
__global__ void k_split_planes(int N, int Np, long Ng, long Ngp, const double* __restrict__ phi,
                               __nv_bfloat16* __restrict__ planes) {
  const long n = (long)Np * Ngp;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const long b = e / ((long)Np * kPK);
    const int k = (int)((e / kPK) % Np);
    const long g = b * kPK + (e % kPK);
    const double x = (k < N && g < Ng) ? phi[(long)k * Ng + g] : 0.0;
    const __nv_bfloat16 h = __double2bfloat16(x);
    planes[e] = h;
    planes[n + e] = __double2bfloat16(x - (double)__bfloat162float(h));
  }
}

// Bt_r[plane][j][k] = Shat_r[k][j] split into bfloat16 hi / lo: 2 dS_kj (k < j), dS_jj (k = j),
// 0 otherwise or past N; dS = S_r - Sa_r (the replica's anchor; float64 in, rounded once per
// plane)
__global__ void k_shat_planes(int N, int Np, const double* __restrict__ S,
                              const double* __restrict__ Sa, long sstride,
                              __nv_bfloat16* __restrict__ bt, const RepCtl* __restrict__ ctl) {
  const int rep = blockIdx.y;
  if (ctl && !ctl[rep].active) return;
  const double* Sr = S + rep * sstride;
  const double* Sref = Sa + rep * sstride;
  const long NpNp = (long)Np * Np;
  __nv_bfloat16* hi = bt + 2 * rep * NpNp;
  __nv_bfloat16* lo = hi + NpNp;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < NpNp;
       e += (long)gridDim.x * blockDim.x) {
    const int j = (int)(e / Np), k = (int)(e % Np);
    double v = 0.0;
    if (j < N && k <= j) {
      const long o = (long)k * N + j;
      v = (k < j) ? 2.0 * (Sr[o] - Sref[o]) : (Sr[o] - Sref[o]);
    }
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi[e] = h;
    lo[e] = __double2bfloat16(v - (double)__bfloat162float(h));
  }
}

// ---- density change on the tensor cores -------------------------------------------------------
// Roles: warp 0 lane 0 issues the TMA copies (Shat's planes once, then 64-orbital chunks of
// 128 points into a ring of `slots`), warp 1 lane 0 issues the MMAs (two tensor-memory
// accumulators of Np columns, alternating between tiles), warps 2..5 (one per TMEM lane
// quadrant, thread <-> point) form drho chunk by chunk.  mbarriers: bfull (Shat loaded),
// full[s] (chunk in slot s), empty[s] (epilogue done with slot s), dch[b][c] (chunk c of the
// tile in accumulator b multiplied), tfree[b] (accumulator b read).  Every wait is bounded; a
// time-out raises the abort flag, the roles leave their loops, and the CTA drains the copies
// and MMAs it issued before it frees tensor memory.
__global__ void __launch_bounds__(kRdThreads, 1)
k_rho_planes(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_bt,
             int N, int Np, int Ng, int nrep, int slots, const double* __restrict__ rho_ref,
             const float* __restrict__ drho_a, double* __restrict__ rho,
             float* __restrict__ drho, const RepCtl* __restrict__ ctl,
             int* status, double* __restrict__ mom, int nx, int ny, int nz, float hgrid) {
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t bfull, full[kRdMaxSlots], empty[kRdMaxSlots];
  __shared__ __align__(8) uint64_t dch[2][kPMaxNp / kPK], tfree[2];
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, issued_n, committed_n;
  __shared__ float momw[4][4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rep = blockIdx.x % nrep;
  const int cta = blockIdx.x / nrep, ncta = gridDim.x / nrep;
  if (ctl && !ctl[rep].active) {   // uniform: nothing to form; moments of this slot zero
    if (mom && tid < 4) mom[(long)(rep * 4 + tid) * ncta + cta] = 0.0;
    return;
  }
  const int C = (Np + kPK - 1) / kPK;                   // orbital chunks
  const int ntiles = (Ng + kPM - 1) / kPM;
  const int ntl = cta < ntiles ? (ntiles - 1 - cta) / ncta + 1 : 0;
  // shared memory: Shat chunks (rows j in [64 c, Np), hi then lo), then the chunk ring
  const uint32_t base = (saddr(smraw) + 1023u) & ~1023u;
  unsigned char* const gbase = smraw + (base - saddr(smraw));
  uint32_t boff[kPMaxNp / kPK];
  uint32_t bbytes = 0;
  for (int c = 0; c < C; ++c) {
    boff[c] = bbytes;
    bbytes += 2u * (uint32_t)(Np - kPK * c) * 128u;
  }
  const uint32_t ring = base + bbytes;
  volatile int* abort_v = &abort_flag;

  if (warp == 1) tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    abort_flag = 0;
    issued_n = 0;
    committed_n = 0;
    mbar_init(&bfull, 1);
    for (int s = 0; s < slots; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 4);
    }
    for (int b = 0; b < 2; ++b) {
      for (int c = 0; c < C; ++c) mbar_init(&dch[b][c], 1);
      mbar_init(&tfree[b], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    // ---- TMA producer ------------------------------------------------------------------------
    if (lane == 0) {
      mbar_expect_tx(saddr(&bfull), bbytes);
      for (int c = 0; c < C; ++c) {
        const int rows = Np - kPK * c;
        for (int j0 = 0; j0 < rows; j0 += 32)   // 32-row boxes: Np - 64 c is a multiple of 32
          for (int pl = 0; pl < 2; ++pl)
            tma_load_3d(base + boff[c] + (uint32_t)(pl * rows + j0) * 128u, &tm_bt, kPK * c,
                        kPK * c + j0, 2 * rep + pl, saddr(&bfull));
      }
      int q = 0;
      for (int i = 0; i < ntl && !*abort_v; ++i) {
        const int x0 = (cta + i * ncta) * kPM;
        for (int c = 0; c < C; ++c, ++q) {
          const int s = q % slots;
          if (q >= slots && !mbar_wait(&empty[s], (uint32_t)(q / slots - 1) & 1u)) {
            *abort_v = 1;
            break;
          }
          const uint32_t dst = ring + (uint32_t)s * kRdSlotB;
          const uint32_t bar = saddr(&full[s]);
          const int b0 = x0 / kPK;                    // the tile's two 64-point blocks
          mbar_expect_tx(bar, (uint32_t)kRdSlotB);
          tma_load_4d(dst, &tm_a, 0, kPK * c, b0, 0, bar);
          tma_load_4d(dst + kPlaneBox, &tm_a, 0, kPK * c, b0 + 1, 0, bar);
          tma_load_4d(dst + 2 * kPlaneBox, &tm_a, 0, kPK * c, b0, 1, bar);
          tma_load_4d(dst + 3 * kPlaneBox, &tm_a, 0, kPK * c, b0 + 1, 1, bar);

          *reinterpret_cast<volatile int*>(&issued_n) = q + 1;
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---- MMA issuer --------------------------------------------------------------------------
    if (lane == 0) {
      bool ok = mbar_wait(&bfull, 0);
      if (!ok) *abort_v = 1;
      int q = 0;
      for (int i = 0; i < ntl && ok && !*abort_v; ++i) {
        const int b = i & 1;
        if (i >= 2 && !mbar_wait(&tfree[b], (uint32_t)((i - 2) >> 1) & 1u)) {
          *abort_v = 1;
          break;
        }
        for (int c = 0; c < C; ++c, ++q) {
          const int s = q % slots;
          if (!mbar_wait(&full[s], (uint32_t)(q / slots) & 1u) || *abort_v) {
            *abort_v = 1;
            ok = false;
            break;
          }
          fence_after();
          const int nc = Np - kPK * c;                  // columns j >= 64 c
          const int nk = min(4, nc / 16);               // 16-orbital steps in this chunk
          const uint32_t idesc = idesc_bf16_major(kPM, nc, 1, 0);
          const uint32_t d = tbase + (uint32_t)(b * kPMaxNp + kPK * c);
          const uint32_t a_hi = ring + (uint32_t)s * kRdSlotB, a_lo = a_hi + 2 * kPlaneBox;
          const uint32_t b_hi = base + boff[c], b_lo = b_hi + (uint32_t)nc * 128u;
          for (int kk = 0; kk < nk; ++kk) {
            const uint64_t ah = sdesc_sw128(a_hi + kk * 2048, kPlaneBox, 1024);
            const uint64_t al = sdesc_sw128(a_lo + kk * 2048, kPlaneBox, 1024);
            const uint64_t bh = sdesc_sw128(b_hi + kk * 32, 16, 1024);
            const uint64_t bl = sdesc_sw128(b_lo + kk * 32, 16, 1024);
            mma_bf16(d, ah, bh, idesc, (c > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d, ah, bl, idesc, 1u);
            mma_bf16(d, al, bh, idesc, 1u);
          }
          mma_commit(&dch[b][c]);
          *reinterpret_cast<volatile int*>(&committed_n) = q + 1;
        }
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: warps 2..5, TMEM lane quadrant wq, point p of the tile ------------------------
    const int wq = warp & 3;
    const int p = 32 * wq + lane;
    const int pb = p >> 6, pp = p & 63;
    const float cx = 0.5f * (float)(nx - 1), cy = 0.5f * (float)(ny - 1), cz = 0.5f * (float)(nz - 1);
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
    int q = 0;
    for (int i = 0; i < ntl; ++i) {
      const int b = i & 1;
      const int g = (cta + i * ncta) * kPM + p;
      // the anchor's density change at this point, loaded ahead of the chunk loop
      const float anc = g < Ng ? __ldg(drho_a + (long)rep * Ng + g) : 0.0f;
      float acc = 0.0f;
      bool ok = true;
      for (int c = 0; c < C; ++c, ++q) {
        const int s = q % slots;
        // the chunk's MMAs are done (their columns are final); the copy into slot s landed
        ok = mbar_wait(&dch[b][c], (uint32_t)(i >> 1) & 1u) &&
             mbar_wait(&full[s], (uint32_t)(q / slots) & 1u) && !*abort_v;
        ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
        if (!ok) break;
        fence_after();
        const unsigned char* sl = gbase + bbytes + (size_t)s * kRdSlotB + pb * kPlaneBox;
        const int nj = min(kPK, Np - kPK * c);
        for (int h = 0; h < 2 && 32 * h < nj; ++h) {   // warp-uniform
          float y[32];
          tmem_ld32(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)(b * kPMaxNp + kPK * c + 32 * h), y);
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            const int k = 32 * h + u;   // orbital row of the chunk
            const int off = k * 128 + (((pp >> 3) ^ (k & 7)) << 4) + ((pp & 7) << 1);
            const float hv = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(sl + off));
            const float lv = __bfloat162float(
                *reinterpret_cast<const __nv_bfloat16*>(sl + 2 * kPlaneBox + off));
            acc = fmaf(hv + lv, y[u], acc);
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      if (!ok) {
        *abort_v = 1;
        break;
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tfree[b]);
      if (g < Ng) {
        acc += anc;   // rho(Sa) - rho_ref
        drho[(long)rep * Ng + g] = acc;
        if (rho) rho[(long)rep * Ng + g] = rho_ref[g] + (double)acc;
        if (mom) {
          const int ix = g % nx, rest = g / nx;
          const float xq = ((float)ix - cx) * hgrid;
          const float yq = ((float)(rest % ny) - cy) * hgrid;
          const float zq = ((float)(rest / ny) - cz) * hgrid;
          m0 += acc;
          m1 = fmaf(acc, xq, m1);
          m2 = fmaf(acc, yq, m2);
          m3 = fmaf(acc, zq, m3);
        }
      }
    }
    if (mom) {
      m0 = warp_sumf(m0);
      m1 = warp_sumf(m1);
      m2 = warp_sumf(m2);
      m3 = warp_sumf(m3);
      if (lane == 0) {
        momw[wq][0] = m0;
        momw[wq][1] = m1;
        momw[wq][2] = m2;
        momw[wq][3] = m3;
      }
    }
  }
  __syncthreads();
  if (mom && tid < 4) {   // fixed order over the four epilogue warps, float64
    double acc = 0.0;
    for (int w = 0; w < 4; ++w) acc += (double)momw[w][tid];
    mom[(long)(rep * 4 + tid) * ncta + cta] = acc;
  }
  if (*abort_v && tid == 0) {
    atomicCAS(status, 0, (int)RMGTD_ETIMEOUT);
    // drain: every issued copy lands and every committed MMA group completes (bounded waits;
    // a completed phase returns at once)
    const int ni = *reinterpret_cast<volatile int*>(&issued_n);
    for (int u = max(0, ni - slots); u < ni; ++u) mbar_wait(&full[u % slots], (uint32_t)(u / slots) & 1u);
    mbar_wait(&bfull, 0);
    const int nc = *reinterpret_cast<volatile int*>(&committed_n);
    if (nc > 0) {
      const int u = nc - 1, i = u / C, c = u % C;
      mbar_wait(&dch[i & 1][c], (uint32_t)(i >> 1) & 1u);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// ---- Gram of the weighted orbitals on the tensor cores ---------------------------------------
// Per replica and grid chunk (split-K), 64-point stages:
//   D_I[i][j] = sum_g (w(g) phi_i(g)) phi_j(g)    (row tile I = 0, 1 of 128 orbitals; j >= 128 I)
// A = w * (hi + lo) of the tile's rows, rounded again into bfloat16 hi / lo by the converter
// warps into one of two operand sets; B = the raw orbital rows 128 I .. Np of the stage (both
// planes, straight from the TMA copy).  Row tile 1 holds Np - 128 rows: its MMAs read 128
// rows from the start of its buffers, and the rows past Np-128 (whatever shared memory follows)
// only reach accumulator rows that are never stored.
// Roles: warp 0 lane 0 issues the copies into a ring of `slots` raw slots (both planes of a
// 64-point block, contiguous, and the stage's weights by bulk copy), warp 1 lane 0 the MMAs
// (accumulator of row tile 0: Np columns at 0; of row tile 1: Np - 128 at Np), the 16 warps
// from 2 on convert (thread: one 16-byte chunk of 8 points in rows r, r + 64, ...) and
// afterwards copy the accumulators to the partials.  mbarriers: full[s] (copies of raw slot s
// landed), rfree[s] (the MMAs reading raw slot s completed), conv[a] (operand set a written,
// one arrival per converter warp), afree[a] (the MMAs reading operand set a completed), accf (all MMAs completed).
// A stage's raw slot is released as soon as its MMAs complete, so `slots` copies stay in flight
// while the converters fill the other operand set.  Every wait is bounded; a time-out raises
// the abort flag and the CTA drains its copies and MMAs before it frees tensor memory.
__host__ __device__ constexpr uint32_t gram_aset_bytes(int Np) {
  return 32768u + (Np > kPM ? 2u * (uint32_t)(Np - kPM) * 128u : 0u);
}
__host__ __device__ constexpr uint32_t gram_raw_bytes(int Np) { return 2u * (uint32_t)Np * 128u + 1024u; }

__global__ void __launch_bounds__(kGpThreads, 1)
k_gram_planes(const __grid_constant__ CUtensorMap tm_b, const float* __restrict__ w,
              const float* __restrict__ w_anchor, int wbulk, int N, int Np, int Ng, int nrep,
              int chunk, int slots, float* __restrict__ part, const RepCtl* __restrict__ ctl,
              int* status) {
  extern __shared__ unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[kGpMaxStages], rfree[kGpMaxStages];
  __shared__ __align__(8) uint64_t conv[2], afree[2], accf;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag, issued_n, committed_n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x, rep = blockIdx.y;
  if (ctl && !ctl[rep].active) return;   // uniform; the reduction skips inactive replicas
  const int TI = Np > kPM ? 2 : 1;
  const int g_beg = split * chunk;
  const int g_end = min(Ng, g_beg + chunk);
  const int nst = g_end > g_beg ? (g_end - g_beg + kPK - 1) / kPK : 0;
  const uint32_t bplane = (uint32_t)Np * 128u;          // one raw plane of a stage
  const uint32_t asetB = gram_aset_bytes(Np);
  const uint32_t a1ofs = 32768u, a1pl = (uint32_t)max(0, Np - kPM) * 128u;
  const uint32_t rawB = gram_raw_bytes(Np), wofs = 2u * bplane;
  // shared memory: operand sets 0, 1, then the raw ring (row tile 1's 128-row reads past its
  // buffers stay inside the allocation)
  const uint32_t base = (saddr(smraw) + 1023u) & ~1023u;
  unsigned char* const gbase = smraw + (base - saddr(smraw));
  const uint32_t ring = base + 2u * asetB;
  volatile int* abort_v = &abort_flag;

  if (warp == 1) tmem_alloc(&tmem_base, 512);
  if (tid == 0) {
    abort_flag = 0;
    issued_n = 0;
    committed_n = 0;
    for (int s = 0; s < slots; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&rfree[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&conv[a], kGConvWarps);
      mbar_init(&afree[a], 1);
    }
    mbar_init(&accf, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = tmem_base;

  if (warp == 0) {
    if (lane == 0) {
      for (int t = 0; t < nst && !*abort_v; ++t) {
        const int s = t % slots;
        if (t >= slots && !mbar_wait(&rfree[s], (uint32_t)(t / slots - 1) & 1u)) {
          *abort_v = 1;
          break;
        }
        const uint32_t dst = ring + (uint32_t)s * rawB;
        const uint32_t bar = saddr(&full[s]);
        const int g0 = g_beg + kPK * t;
        // the weights by bulk copy (rows 16-byte aligned: Ng a multiple of 4); points of the
        // stage past Ng are not copied and are masked by the converters
        const uint32_t wb = wbulk ? 4u * (uint32_t)min(kPK, Ng - g0) : 0u;
        mbar_expect_tx(bar, 2u * bplane + (w_anchor ? 2u : 1u) * wb);
        tma_load_4d(dst, &tm_b, 0, 0, g0 / kPK, 0, bar);
        tma_load_4d(dst + bplane, &tm_b, 0, 0, g0 / kPK, 1, bar);
        if (wb) {
          bulk_g2s_1d(dst + wofs, w + (long)rep * Ng + g0, wb, bar);
          if (w_anchor) bulk_g2s_1d(dst + wofs + 256u, w_anchor + (long)rep * Ng + g0, wb, bar);
        }
        *reinterpret_cast<volatile int*>(&issued_n) = t + 1;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int t = 0; t < nst; ++t) {
        const int s = t % slots, a = t & 1;
        if (!mbar_wait(&conv[a], (uint32_t)(t >> 1) & 1u) || *abort_v) {
          *abort_v = 1;
          ok = false;
          break;
        }
        fence_after();
        const uint32_t ab = base + (uint32_t)a * asetB, rb = ring + (uint32_t)s * rawB;
        for (int I = 0; I < TI; ++I) {
          const int nI = Np - kPM * I;
          const uint32_t idesc = idesc_bf16_major(kPM, nI, 0, 0);
          const uint32_t d = tbase + (uint32_t)(I ? Np : 0);
          const uint32_t a_hi = ab + (I ? a1ofs : 0u), a_lo = a_hi + (I ? a1pl : 16384u);
          const uint32_t b_hi = rb + (uint32_t)(kPM * I) * 128u, b_lo = b_hi + bplane;
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ah = sdesc_sw128(a_hi + kk * 32, 16, 1024);
            const uint64_t al = sdesc_sw128(a_lo + kk * 32, 16, 1024);
            const uint64_t bh = sdesc_sw128(b_hi + kk * 32, 16, 1024);
            const uint64_t bl = sdesc_sw128(b_lo + kk * 32, 16, 1024);
            mma_bf16(d, ah, bh, idesc, (t > 0 || kk > 0) ? 1u : 0u);
            mma_bf16(d, ah, bl, idesc, 1u);
            mma_bf16(d, al, bh, idesc, 1u);
          }
        }
        mma_commit(&rfree[s]);
        mma_commit(&afree[a]);
        *reinterpret_cast<volatile int*>(&committed_n) = t + 1;
      }
      if (ok && nst > 0) mma_commit(&accf);
    }
    __syncwarp();
  } else {
    // ---- converters: A = w * (hi + lo) of rows 0 .. Np-1 into operand set t & 1 ---------------
    // thread: logical 16-byte chunk c (points 8 c .. 8 c + 7) of rows r0, r0 + 64, ...; rows
    // 64 apart share the swizzle phase, so every offset is a per-thread constant plus 8 KB steps
    const int ct = tid - 64;                 // 0 .. 32 kGConvWarps - 1
    const int c = ct & 7, r0 = ct >> 3;
    constexpr int kRowStep = 4 * kGConvWarps;  // 64 rows per pass
    static_assert(kRowStep % 8 == 0, "rows of a thread must share the swizzle phase");
    const uint32_t sw = (uint32_t)((c ^ (r0 & 7)) << 4);
    const int nrow = r0 < Np ? (Np - 1 - r0) / kRowStep + 1 : 0;   // <= 4 (Np <= 256)
    const float* wr = w + (long)rep * Ng;
    const float* war = w_anchor ? w_anchor + (long)rep * Ng : nullptr;
    for (int t = 0; t < nst; ++t) {
      const int s = t % slots, a = t & 1;
      bool ok = mbar_wait(&full[s], (uint32_t)(t / slots) & 1u);
      if (ok && t >= 2) ok = mbar_wait(&afree[a], (uint32_t)((t >> 1) - 1) & 1u);
      if (!ok || *abort_v) {
        *abort_v = 1;
        break;
      }
      const int g0 = g_beg + kPK * t + 8 * c;
      const uint32_t rs = ring + (uint32_t)s * rawB;    // shared addresses
      const uint32_t as = base + (uint32_t)a * asetB;
      float wv[8];
      if (wbulk && g0 + 8 <= g_end) {
        const float4 w0 = lds_f4(rs + wofs + 32u * c), w1 = lds_f4(rs + wofs + 32u * c + 16u);
        wv[0] = w0.x; wv[1] = w0.y; wv[2] = w0.z; wv[3] = w0.w;
        wv[4] = w1.x; wv[5] = w1.y; wv[6] = w1.z; wv[7] = w1.w;
        if (war) {
          const float4 v0 = lds_f4(rs + wofs + 256u + 32u * c), v1 = lds_f4(rs + wofs + 272u + 32u * c);
          wv[0] -= v0.x; wv[1] -= v0.y; wv[2] -= v0.z; wv[3] -= v0.w;
          wv[4] -= v1.x; wv[5] -= v1.y; wv[6] -= v1.z; wv[7] -= v1.w;
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float v = 0.0f;
          if (g0 + e < g_end) {
            if (wbulk)
              v = war ? lds_f(rs + wofs + 4u * (8 * c + e)) - lds_f(rs + wofs + 256u + 4u * (8 * c + e))
                      : lds_f(rs + wofs + 4u * (8 * c + e));
            else
              v = war ? __ldg(wr + g0 + e) - __ldg(war + g0 + e) : __ldg(wr + g0 + e);
          }
          wv[e] = v;
        }
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (k < nrow) {
          const int R = r0 + kRowStep * k;
          const uint32_t off = (uint32_t)R * 128u + sw;
          const uint4 h4 = lds_u4(rs + off);
          const uint4 l4 = lds_u4(rs + bplane + off);
          const uint32_t hv[4] = {h4.x, h4.y, h4.z, h4.w}, lv[4] = {l4.x, l4.y, l4.z, l4.w};
          uint32_t oh[4], ol[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float x0 = fmaf(bf_lo(hv[u]), wv[2 * u], bf_lo(lv[u]) * wv[2 * u]);
            const float x1 = fmaf(bf_hi(hv[u]), wv[2 * u + 1], bf_hi(lv[u]) * wv[2 * u + 1]);
            split2(x0, x1, oh[u], ol[u]);
          }
          // row R of tile R / 128 at the same swizzled position (128 I is a multiple of 8)
          const uint32_t ah = R < kPM ? as + off : as + a1ofs + off - (uint32_t)kPM * 128u;
          const uint32_t al = ah + (R < kPM ? 16384u : a1pl);
          sts_u4(ah, make_uint4(oh[0], oh[1], oh[2], oh[3]));
          sts_u4(al, make_uint4(ol[0], ol[1], ol[2], ol[3]));
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[a]);
    }
    // ---- epilogue: accumulators -> partials (rows of the upper block triangle) ---------------
    bool ok = !*abort_v;
    if (ok && nst > 0) ok = mbar_wait(&accf, 0);
    ok = __all_sync(0xffffffffu, ok);   // tcgen05.ld below is warp-collective
    if (!ok) *abort_v = 1;
    fence_after();
    // warps sharing a TMEM lane quadrant (warp mod 4) split the 32-column groups
    const int wq = warp & 3, grp = (warp - 2) >> 2;
    if (ok) {
      for (int I = 0; I < TI; ++I) {
        const int row = kPM * I + 32 * wq + lane;
        const int nI = Np - kPM * I;
        float* prow = part + ((long)(split * nrep + rep) * Np + row) * Np + kPM * I;
        for (int m = grp; m < nI / 32; m += kGConvWarps / 4) {
          float y[32];
          if (nst > 0) {
            tmem_ld32(tbase + ((uint32_t)(wq * 32) << 16) + (uint32_t)((I ? Np : 0) + 32 * m), y);
          } else {
#pragma unroll
            for (int u = 0; u < 32; ++u) y[u] = 0.0f;
          }
          if (row < Np) {
#pragma unroll
            for (int u = 0; u < 32; u += 4)
              *reinterpret_cast<float4*>(prow + 32 * m + u) =
                  make_float4(y[u], y[u + 1], y[u + 2], y[u + 3]);
          }
        }
      }
    }
  }
  __syncthreads();
  if (*abort_v && tid == 0) {
    atomicCAS(status, 0, (int)RMGTD_ETIMEOUT);
    const int ni = *reinterpret_cast<volatile int*>(&issued_n);
    for (int u = max(0, ni - slots); u < ni; ++u)
      mbar_wait(&full[u % slots], (uint32_t)(u / slots) & 1u);
    // the last commit covers every MMA issued before it
    const int nc = *reinterpret_cast<volatile int*>(&committed_n);
    if (nc > 0) mbar_wait(&rfree[(nc - 1) % slots], (uint32_t)((nc - 1) / slots) & 1u);
  }
  (void)N;
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tbase, 512);
  }
}

}  // namespace tc

namespace {

// 4-D bfloat16 tensor map of the orbital planes [2][nblk][Np][64]: dims {64, Np, nblk, 2},
// box {box_x, box_y, 1, 1}, the given swizzle, zero fill out of bounds (rows past Np too)
bool encode_blocked_planes(void* map, const void* base, long Np, long nblk, int box_x,
                           int box_y, CUtensorMapSwizzle swz) {
  const EncodeTiledFn f = tensor_map_encoder();
  if (!f) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)tc::kPK, (cuuint64_t)Np, (cuuint64_t)nblk, 2};
  const cuuint64_t strides[3] = {(cuuint64_t)tc::kPK * 2, (cuuint64_t)Np * tc::kPK * 2,
                                 (cuuint64_t)nblk * Np * tc::kPK * 2};
  const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return f(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4,
           const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D bfloat16 tensor map: dims {x, y, z} with row stride x_stride elements and plane stride
// z_stride elements, box {64, box_y, 1}, 128-byte swizzle, zero fill out of bounds
bool encode_planes(void* map, const void* base, long x, long y, long z, long x_stride,
                   long z_stride, int box_y) {
  const EncodeTiledFn f = tensor_map_encoder();
  if (!f) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)x, (cuuint64_t)y, (cuuint64_t)z};
  const cuuint64_t strides[2] = {(cuuint64_t)x_stride * 2, (cuuint64_t)z_stride * 2};
  const cuuint32_t box[3] = {(cuuint32_t)tc::kPK, (cuuint32_t)box_y, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return f(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
           const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t rho_planes_smem(int Np, int slots) {
  size_t b = 0;
  for (int c = 0; c * tc::kPK < Np; ++c) b += 2u * (size_t)(Np - tc::kPK * c) * 128u;
  return 1024 + b + (size_t)slots * tc::kRdSlotB;
}

size_t gram_planes_smem(int Np, int slots) {
  return 1024 + 2 * (size_t)tc::gram_aset_bytes(Np) + (size_t)slots * tc::gram_raw_bytes(Np);
}

}  // namespace

// Orbital planes of the mixed path (set-up): allocated and filled when 32 < N <= 256 and the
// grid and sizes suit the tensor maps; otherwise nothing happens (the caller keeps the other
// kernels).  Returns the status.
int planes_setup(rmgtd_ctx* ctx) {
  using namespace tc;
  const int N = ctx->N;
  const int Np = ((N + 31) / 32) * 32;
  if (N <= 32 || Np > kPMaxNp || ctx->Ng >= (1l << 31) - 256 || !tensor_map_encoder())
    return RMGTD_OK;
  if (rho_planes_smem(Np, 2) > (size_t)kSmemLimit || gram_planes_smem(Np, 1) > (size_t)kSmemLimit)
    return RMGTD_OK;
  const long Ngp = ((ctx->Ng + kPK - 1) / kPK) * kPK;
  const size_t pbytes = 2 * sizeof(__nv_bfloat16) * (size_t)Np * Ngp;
  ctx->phi_pl = (__nv_bfloat16*)dev_alloc(ctx, pbytes);
  ctx->bt_pl = (__nv_bfloat16*)dev_alloc(ctx, 2 * sizeof(__nv_bfloat16) * (size_t)Np * Np * ctx->nrep);
  if (!ctx->phi_pl || !ctx->bt_pl) return set_error(ctx, RMGTD_ENOMEM, "orbital planes");
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->bt_pl, 0, 2 * sizeof(__nv_bfloat16) * (size_t)Np * Np * ctx->nrep,
                                  ctx->stream));
  const long n = (long)Np * Ngp;
  const int blocks = (int)std::max<long>(1, std::min<long>(ceil_div(n, 256), 16L * ctx->num_sms));
  k_split_planes<<<blocks, 256, 0, ctx->stream>>>(N, Np, ctx->Ng, Ngp, ctx->phi, ctx->phi_pl);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_split_planes");
  if (!encode_blocked_planes(ctx->tm_pa, ctx->phi_pl, Np, Ngp / kPK, kPK, kPK,
                             CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_blocked_planes(ctx->tm_pb, ctx->phi_pl, Np, Ngp / kPK, kPK, Np,
                             CU_TENSOR_MAP_SWIZZLE_128B) ||
      !encode_planes(ctx->tm_bt, ctx->bt_pl, Np, Np, 2L * ctx->nrep, Np, (long)Np * Np, 32)) {
    dev_free(ctx, ctx->phi_pl);
    dev_free(ctx, ctx->bt_pl);
    ctx->phi_pl = nullptr;
    ctx->bt_pl = nullptr;
    return RMGTD_OK;
  }
  const size_t msz = sizeof(double) * (size_t)N * N * ctx->nrep;
  const size_t fsz = sizeof(float) * (size_t)ctx->Ng * ctx->nrep;
  ctx->Sa = (double*)dev_alloc(ctx, msz);
  ctx->Ha = (double*)dev_alloc(ctx, msz);
  ctx->rho_a32 = (float*)dev_alloc(ctx, fsz);
  ctx->dv_a32 = (float*)dev_alloc(ctx, fsz);
  if (!ctx->Sa || !ctx->Ha || !ctx->rho_a32 || !ctx->dv_a32)
    return set_error(ctx, RMGTD_ENOMEM, "orbital-plane anchors");
  ctx->Np_pl = Np;
  ctx->Ngp_pl = Ngp;
  return RMGTD_OK;
}

int planes_anchor_reset(rmgtd_ctx* ctx) {
  if (!ctx->phi_pl) return RMGTD_OK;
  const size_t NN = (size_t)ctx->N * ctx->N;
  for (int r = 0; r < ctx->nrep; ++r) {
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Sa + r * NN, ctx->Sref, sizeof(double) * NN,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
    RMGTD_CUDA(ctx, cudaMemcpyAsync(ctx->Ha + r * NN, ctx->Href, sizeof(double) * NN,
                                    cudaMemcpyDeviceToDevice, ctx->stream));
  }
  const size_t fsz = sizeof(float) * (size_t)ctx->Ng * ctx->nrep;
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->rho_a32, 0, fsz, ctx->stream));
  RMGTD_CUDA(ctx, cudaMemsetAsync(ctx->dv_a32, 0, fsz, ctx->stream));
  return RMGTD_OK;
}

namespace tc {

// After a step: when it completed for every replica (k_step_end's condition: no earlier
// failure in this call, device status clear, every replica's status clear) the anchors move
// to the new state: Sa <- S0 (= the final P_1), Ha <- H0 (= H of the final pass),
// rho_a <- drho and Va <- dV of that pass.
__global__ void k_anchor_update(long nm, long ng, const double* __restrict__ S0,
                                const double* __restrict__ H0, const float* __restrict__ drho,
                                const float* __restrict__ dv, double* __restrict__ Sa,
                                double* __restrict__ Ha, float* __restrict__ rho_a,
                                float* __restrict__ dv_a, const RepCtl* __restrict__ ctl,
                                int nrep, const int* failed, const int* status) {
  if (*failed || *status != 0) return;
  for (int r = 0; r < nrep; ++r)
    if (ctl[r].status != 0) return;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < nm; e += stride) {
    Sa[e] = S0[e];
    Ha[e] = H0[e];
  }
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < ng; e += stride) {
    rho_a[e] = drho[e];
    dv_a[e] = dv[e];
  }
}

}  // namespace tc

int planes_anchor_update(rmgtd_ctx* ctx) {
  if (!ctx->phi_pl || !ctx->mixed) return RMGTD_OK;
  const long nm = (long)ctx->nrep * ctx->N * ctx->N, ng = (long)ctx->nrep * ctx->Ng;
  const int blocks = (int)std::max<long>(1, std::min<long>(ceil_div(ng, 256), 4L * ctx->num_sms));
  tc::k_anchor_update<<<blocks, 256, 0, ctx->stream>>>(nm, ng, ctx->S0, ctx->H0, ctx->drho32,
                                                       ctx->dv32, ctx->Sa, ctx->Ha, ctx->rho_a32,
                                                       ctx->dv_a32, ctx->ctl, ctx->nrep,
                                                       ctx->failed, ctx->status);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_anchor_update");
  return RMGTD_OK;
}

// Density change of the mixed path through the orbital planes; returns 1 when the planes
// are not set up (the caller runs the other kernels), else the status.
int rho_planes(rmgtd_ctx* ctx, const double* S, double* rho, float* drho, const RepCtl* ctl,
               int nrep) {
  using namespace tc;
  if (!ctx->phi_pl) return 1;
  const int N = ctx->N, Np = ctx->Np_pl;
  const long NpNp = (long)Np * Np;
  k_shat_planes<<<dim3(std::max(1, (int)std::min<long>(ceil_div(NpNp, 256), 256)), nrep), 256, 0,
                  ctx->stream>>>(N, Np, S, ctx->Sa, (long)N * N, ctx->bt_pl, ctl);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_shat_planes");
  int slots = kRdMaxSlots;
  while (slots > 2 && rho_planes_smem(Np, slots) > (size_t)kSmemLimit) --slots;
  const size_t smem = rho_planes_smem(Np, slots);
  // the attribute belongs to the function (process-wide, shared by every context): only ever
  // raise it (a smaller N may need more shared memory: more slots fit)
  if (ctx->rho_pl_attr < (int)smem) {
    cudaFuncAttributes fa;
    RMGTD_CUDA(ctx, cudaFuncGetAttributes(&fa, k_rho_planes));
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
      RMGTD_CUDA(ctx, cudaFuncSetAttribute(k_rho_planes, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
    ctx->rho_pl_attr = (int)smem;
  }
  const int ncta = std::max(1, ctx->num_sms / nrep);
  const int grid = ncta * nrep;
  double* mom = nullptr;
  if (ctx->rho_mom && (long)4 * nrep * ncta <= ctx->rho_mom_cap) mom = ctx->rho_mom;
  CUtensorMap ta, tb;
  memcpy(&ta, ctx->tm_pa, sizeof(ta));
  memcpy(&tb, ctx->tm_bt, sizeof(tb));
  k_rho_planes<<<grid, kRdThreads, smem, ctx->stream>>>(
      ta, tb, N, Np, (int)ctx->Ng, nrep, slots, ctx->rho_ref, ctx->rho_a32, rho, drho, ctl,
      ctx->status, mom,
      ctx->nx, ctx->ny, ctx->nz, (float)ctx->h);
  ctx->rho_mom_blocks = mom ? ncta : 0;
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_rho_planes");
  return RMGTD_OK;
}

// Gram partials of the mixed path through the orbital planes (layout of k_gram32's); returns
// 1 when the planes are not set up, else the status.  chunk must be a multiple of 64.
int gram_planes(rmgtd_ctx* ctx, const float* w, const float* w_anchor, int nw, float* part,
                int nsplit, int chunk, const RepCtl* ctl) {
  using namespace tc;
  if (!ctx->phi_pl || chunk % kPK) return 1;
  const int Np = ctx->Np_pl;
  int stages = kGpMaxStages;
  while (stages > 1 && gram_planes_smem(Np, stages) > (size_t)kSmemLimit) --stages;
  const size_t smem = gram_planes_smem(Np, stages);
  if (ctx->gram_pl_attr < (int)smem) {   // process-wide attribute: only ever raise it
    cudaFuncAttributes fa;
    RMGTD_CUDA(ctx, cudaFuncGetAttributes(&fa, k_gram_planes));
    if ((size_t)fa.maxDynamicSharedSizeBytes < smem)
      RMGTD_CUDA(ctx, cudaFuncSetAttribute(k_gram_planes,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ctx->gram_pl_attr = (int)smem;
  }
  CUtensorMap tb;
  memcpy(&tb, ctx->tm_pb, sizeof(tb));
  k_gram_planes<<<dim3(nsplit, nw), kGpThreads, smem, ctx->stream>>>(
      tb, w, w_anchor, ctx->Ng % 4 == 0 ? 1 : 0, ctx->N, Np, (int)ctx->Ng, nw, chunk, stages,
      part, ctl, ctx->status);
  ++ctx->launches;
  RMGTD_LAUNCH(ctx, "k_gram_planes");
  return RMGTD_OK;
}

}  // namespace rmgtd
