// Register-resident DFT codelets and the two-stage line FFT of the fast local-potential path.
//
// A line of length N = R1 * R2 is transformed by a group of G = max(R1, R2) threads with one
// shared-memory exchange (Cooley-Tukey with the index maps n = R2 n1 + n2, k = k1 + R1 k2):
//
//   fft2_nat: thread t < R2 holds x[R2 n1 + t] (n1 < R1)  ->  thread t < R1 holds X[t + R1 k2] (k2 < R2)
//   fft2_rev: thread t < R1 holds x[t + R1 k2] (k2 < R2)  ->  thread t < R2 holds X[t + R2 m1] (m1 < R1)
//
// so a transform taken with fft2_nat can be followed by a pointwise product and a transform of
// the opposite sign with fft2_rev, with no reordering in between.  The R-point codelets are
// radix 2, 3, 4, 5 written out, and composite sizes split once more in registers; their twiddles
// are compile-time constants from the exact-argument series in CxTrig.  The inter-stage twiddles
// w^(t k) (run-time t) come from a per-size table e^{-2 pi i j / N} kept in shared memory.
#pragma once

#include <cuda_runtime.h>

#include "warp_fft.cuh"

namespace hpsi {

// cos(2 pi k / n) and sin(2 pi k / n) evaluated at compile time: the argument is reduced exactly
// with integer arithmetic to theta in [0, pi/4] and the Taylor series of sin and cos is summed.
struct CxTrig {
  static constexpr double kPi = 3.14159265358979323846264338327950288;
  __host__ __device__ static constexpr double sin_s(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int i = 1; i <= 13; ++i) {
      term *= -x2 / (double)((2 * i) * (2 * i + 1));
      sum += term;
    }
    return sum;
  }
  __host__ __device__ static constexpr double cos_s(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int i = 1; i <= 13; ++i) {
      term *= -x2 / (double)((2 * i - 1) * (2 * i));
      sum += term;
    }
    return sum;
  }
  // component 0: cos, 1: sin of 2 pi k / n
  __host__ __device__ static constexpr double cs(long k, long n, int which) {
    long kk = k % n;
    if (kk < 0) kk += n;
    const long o = (8 * kk) / n, r = (8 * kk) % n;   // angle = (pi/4) (o + r/n)
    double c = 0.0, s = 0.0;
    long q = 0;
    if ((o & 1) == 0) {                                // o pi/4 + theta
      const double th = (kPi / 4.0) * (double)r / (double)n;
      c = cos_s(th);
      s = sin_s(th);
      q = o / 2;
    } else {                                           // (o + 1) pi/4 - theta'
      const double th = (kPi / 4.0) * (double)(n - r) / (double)n;
      c = cos_s(th);
      s = -sin_s(th);
      q = ((o + 1) / 2) % 4;
    }
    // rotate (c, s) by q quarter turns
    double rc = c, rs = s;
    if (q == 1) { rc = -s; rs = c; }
    else if (q == 2) { rc = -c; rs = -s; }
    else if (q == 3) { rc = s; rs = -c; }
    return which == 0 ? rc : rs;
  }
};

template <int N> struct CxTable {
  double c[N > 0 ? N : 1];
  double s[N > 0 ? N : 1];
  __host__ __device__ constexpr CxTable() : c(), s() {
    for (int k = 0; k < N; ++k) {
      c[k] = CxTrig::cs(k, N, 0);
      s[k] = CxTrig::cs(k, N, 1);
    }
  }
};

// v * e^{DIR 2 pi i e / R} with e a compile-time exponent after unrolling
template <int R, int DIR, typename V>
__device__ __forceinline__ V twiddle_c(V v, int e) {
  using T = typename Real<V>::type;
  constexpr CxTable<R> tab{};
  const int m = e % R;
  if (m == 0) return v;
  if ((4 * m) % R == 0) {
    const int q = (4 * m) / R;                     // quarter turns
    V r;
    if (q == 2) { r.x = -v.x; r.y = -v.y; return r; }
    // (q == 1 and DIR > 0) or (q == 3 and DIR < 0): multiply by +i
    if ((q == 1) == (DIR > 0)) { r.x = -v.y; r.y = v.x; } else { r.x = v.y; r.y = -v.x; }
    return r;
  }
  const T c = (T)tab.c[m], s = (T)(DIR > 0 ? tab.s[m] : -tab.s[m]);
  V r;
  r.x = v.x * c - v.y * s;
  r.y = v.x * s + v.y * c;
  return r;
}

template <int R, int DIR, typename V> struct Cdl;
template <int DIR, typename V> struct Cdl<2, DIR, V> { static __device__ __forceinline__ void run(V* x) { Dft<2, DIR, V>::run(x); } };
template <int DIR, typename V> struct Cdl<3, DIR, V> { static __device__ __forceinline__ void run(V* x) { Dft<3, DIR, V>::run(x); } };
template <int DIR, typename V> struct Cdl<4, DIR, V> { static __device__ __forceinline__ void run(V* x) { Dft<4, DIR, V>::run(x); } };
template <int DIR, typename V> struct Cdl<5, DIR, V> { static __device__ __forceinline__ void run(V* x) { Dft<5, DIR, V>::run(x); } };

// R = A * B in registers: x[B n1 + n2] -> X[k1 + A k2]
template <int A, int B, int DIR, typename V> struct CdlAB {
  static __device__ __forceinline__ void run(V* x) {
    constexpr int R = A * B;
    V y[R];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
      V t[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n1] = x[B * n1 + n2];
      Cdl<A, DIR, V>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) y[n2 * A + k1] = twiddle_c<R, DIR>(t[k1], n2 * k1);
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      V t[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2 * A + k1];
      Cdl<B, DIR, V>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = t[k2];
    }
  }
};
template <int DIR, typename V> struct Cdl<6, DIR, V> : CdlAB<2, 3, DIR, V> {};
template <int DIR, typename V> struct Cdl<8, DIR, V> : CdlAB<2, 4, DIR, V> {};
template <int DIR, typename V> struct Cdl<9, DIR, V> : CdlAB<3, 3, DIR, V> {};
template <int DIR, typename V> struct Cdl<10, DIR, V> : CdlAB<2, 5, DIR, V> {};
template <int DIR, typename V> struct Cdl<12, DIR, V> : CdlAB<3, 4, DIR, V> {};
template <int DIR, typename V> struct Cdl<15, DIR, V> : CdlAB<3, 5, DIR, V> {};
template <int DIR, typename V> struct Cdl<16, DIR, V> : CdlAB<4, 4, DIR, V> {};

// v * (table entry j)^(DIR): table holds e^{-2 pi i j / N}
template <int DIR, typename V>
__device__ __forceinline__ V twiddle_t(V v, V w) {
  if (DIR > 0) w.y = -w.y;
  V r;
  r.x = v.x * w.x - v.y * w.y;
  r.y = v.x * w.y + v.y * w.x;
  return r;
}

// Entries of one group's exchange buffer: rows padded by one element so that the row reads of the
// second stage fall in different shared-memory banks.
template <int R1, int R2> struct Xch {
  static constexpr int size = (R1 * (R2 + 1) > R2 * (R1 + 1) ? R1 * (R2 + 1) : R2 * (R1 + 1));
};

// See the file comment.  reg has max(R1, R2) entries; xb is the group's exchange buffer of
// Xch<R1, R2>::size entries; tw the N-entry table.  Every lane of the warp must call (the
// exchange uses __syncwarp).
template <int R1, int R2, int DIR, typename V>
__device__ __forceinline__ void fft2_nat(V* reg, V* xb, const V* tw, int t, bool active) {
  if (active && t < R2) {
    Cdl<R1, DIR, V>::run(reg);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) xb[k1 * (R2 + 1) + t] = k1 == 0 ? reg[0] : twiddle_t<DIR>(reg[k1], tw[t * k1]);
  }
  __syncwarp();
  if (active && t < R1) {
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) reg[n2] = xb[t * (R2 + 1) + n2];
    Cdl<R2, DIR, V>::run(reg);
  }
  __syncwarp();
}

template <int R1, int R2, int DIR, typename V>
__device__ __forceinline__ void fft2_rev(V* reg, V* xb, const V* tw, int t, bool active) {
  if (active && t < R1) {
    Cdl<R2, DIR, V>::run(reg);
#pragma unroll
    for (int m2 = 0; m2 < R2; ++m2) xb[m2 * (R1 + 1) + t] = m2 == 0 ? reg[0] : twiddle_t<DIR>(reg[m2], tw[t * m2]);
  }
  __syncwarp();
  if (active && t < R2) {
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) reg[k1] = xb[t * (R1 + 1) + k1];
    Cdl<R1, DIR, V>::run(reg);
  }
  __syncwarp();
}

}  // namespace hpsi
