// Division of 0 <= x < 2^31 by a fixed d >= 1 with one multiply-high (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994): with l = ceil(log2 d)
// and m = ceil(2^(31+l) / d), floor(x / d) = (x m) >> (31 + l) exactly, because
// 0 <= x m / 2^(31+l) - x / d < x / 2^(31+l) < 2^-l <= 1 / d.  Host and device.
#pragma once

#ifdef __CUDACC__
#define RMGTD_HD __host__ __device__ __forceinline__
#else
#define RMGTD_HD inline
#endif

namespace rmgtd {

struct FastDiv {
  unsigned long long m;
  int s;
  int d;
};

inline FastDiv make_fastdiv(int d) {
  int l = 0;
  while ((1ll << l) < d) ++l;
  FastDiv f;
  f.s = 31 + l;
  f.m = ((1ull << f.s) + (unsigned long long)d - 1) / (unsigned long long)d;
  f.d = d;
  return f;
}

RMGTD_HD int fdiv(int x, const FastDiv& f) {
  return (int)(((unsigned long long)(unsigned)x * f.m) >> f.s);
}

}  // namespace rmgtd
