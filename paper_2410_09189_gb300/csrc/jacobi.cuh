// Symmetric eigen-decomposition of a small float64 matrix by parallel cyclic Jacobi rotations
// inside one thread block (round-robin pairing: N/2 disjoint rotations per round, applied to
// the rows, then to the columns and to the accumulated eigenvectors), at most 40 sweeps,
// stopping when the off-diagonal squared norm is below 1e-28 of the total.  A (N x N,
// row-major, overwritten by the rotated matrix: its diagonal holds the eigenvalues) and V (the
// identity on entry, the eigenvectors as columns on exit) live in global or shared memory;
// pp/qq/cc/ss hold N/2 + 1 entries (N <= 1024); sh is block_sum scratch.
#pragma once

#include "rmgtd_internal.cuh"

namespace rmgtd {

__device__ inline void jacobi_sweeps(int N, double* A, double* V, int* pp, int* qq, double* cc,
                                     double* ss, double* sh, volatile double* stop_flag) {
  const long NN = (long)N * N;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int n2 = N + (N & 1);
  const int np = n2 / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (long e = tid; e < NN; e += nt) {
      const double a = A[e];
      tot += a * a;
      if ((e / N) != (e % N)) off += a * a;
    }
    off = block_sum(off, sh);
    __syncthreads();
    tot = block_sum(tot, sh);
    if (tid == 0) *stop_flag = (off <= 1e-28 * tot) ? 1.0 : 0.0;
    __syncthreads();
    if (*stop_flag != 0.0) break;
    for (int r = 0; r < n2 - 1; ++r) {
      for (int i = tid; i < np; i += nt) {
        const int a0 = (i == 0) ? 0 : ((i - 1 + r) % (n2 - 1)) + 1;
        const int b0 = ((n2 - 2 - i + r) % (n2 - 1)) + 1;
        int p = min(a0, b0), q = max(a0, b0);
        double c = 1.0, sn = 0.0;
        if (q < N) {
          const double apq = A[(long)p * N + q];
          if (fabs(apq) > 1e-300) {
            const double tau = (A[(long)q * N + q] - A[(long)p * N + p]) / (2.0 * apq);
            double t;
            if (fabs(tau) > 1e150)
              t = 0.5 / tau;
            else
              t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
        } else {
          p = q = -1;
        }
        pp[i] = p;
        qq[i] = q;
        cc[i] = c;
        ss[i] = sn;
      }
      __syncthreads();
      for (long e = tid; e < (long)np * N; e += nt) {  // rows: A <- J^T A
        const int i = (int)(e / N), k = (int)(e % N);
        const int p = pp[i], q = qq[i];
        if (p < 0) continue;
        const double ap = A[(long)p * N + k], aq = A[(long)q * N + k];
        A[(long)p * N + k] = cc[i] * ap - ss[i] * aq;
        A[(long)q * N + k] = ss[i] * ap + cc[i] * aq;
      }
      __syncthreads();
      for (long e = tid; e < (long)np * N; e += nt) {  // columns: A <- A J, V <- V J
        const int i = (int)(e / N), k = (int)(e % N);
        const int p = pp[i], q = qq[i];
        if (p < 0) continue;
        const double ap = A[(long)k * N + p], aq = A[(long)k * N + q];
        A[(long)k * N + p] = cc[i] * ap - ss[i] * aq;
        A[(long)k * N + q] = ss[i] * ap + cc[i] * aq;
        const double vp = V[(long)k * N + p], vq = V[(long)k * N + q];
        V[(long)k * N + p] = cc[i] * vp - ss[i] * vq;
        V[(long)k * N + q] = ss[i] * vp + cc[i] * vq;
      }
      __syncthreads();
    }
  }
}

}  // namespace rmgtd
