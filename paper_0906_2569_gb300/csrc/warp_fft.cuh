// Warp-level mixed-radix FFT on a line held in shared memory.
//
// Self-sorting (Stockham) decomposition: for each radix pass R with Ns = product of the earlier
// radices, butterfly j < n/R reads x[j + r n/R], multiplies input r by w^{r (j mod Ns)} with
// w = e^{-+2 pi i / (Ns R)}, takes an R-point DFT in registers and writes the results to
// (j div Ns) Ns R + (j mod Ns) + r Ns.  A pass reads all its inputs into registers before any
// lane writes, so the line is transformed in place; one warp owns one line, so passes are
// separated by __syncwarp only.  Twiddles come from a host-made table (host sin/cos); the
// constants of the radix-3 and radix-5 kernels are the algebraic values of cos/sin(2 pi k/R).
//
// DIR = +1: out[j] = sum_m in[m] e^{+2 pi i m j / n}   (G -> r, no normalisation)
// DIR = -1: out[m] = sum_j in[j] e^{-2 pi i m j / n}   (r -> G, no normalisation)
#pragma once

#include <cuda_runtime.h>

#include "hpsi_internal.h"

namespace hpsi {

template <typename T> struct Cx;
template <> struct Cx<double> { using type = double2; };
template <> struct Cx<float> { using type = float2; };

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// i * DIR * a
template <int DIR, typename V>
__device__ __forceinline__ V cmuli(V a) {
  V r;
  if (DIR > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}
template <typename V> __device__ __forceinline__ V czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

template <typename V> struct Real;
template <> struct Real<double2> { using type = double; };
template <> struct Real<float2> { using type = float; };

// cos(2 pi/5), cos(4 pi/5), sin(2 pi/5), sin(4 pi/5), sin(2 pi/3)
#define HPSI_C5_1 0.30901699437494742410
#define HPSI_C5_2 -0.80901699437494742410
#define HPSI_S5_1 0.95105651629515357212
#define HPSI_S5_2 0.58778525229247312917
#define HPSI_S3 0.86602540378443864676

template <int R, int DIR, typename V> struct Dft;

template <int DIR, typename V> struct Dft<2, DIR, V> {
  static __device__ __forceinline__ void run(V* v) {
    V a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int DIR, typename V> struct Dft<3, DIR, V> {
  static __device__ __forceinline__ void run(V* v) {
    using T = typename Real<V>::type;
    V t1 = cadd(v[1], v[2]);
    V t2 = csub(v[0], cscale(t1, (T)0.5));
    V t3 = cmuli<DIR>(cscale(csub(v[1], v[2]), (T)HPSI_S3));
    v[0] = cadd(v[0], t1);
    v[1] = cadd(t2, t3);
    v[2] = csub(t2, t3);
  }
};

template <int DIR, typename V> struct Dft<4, DIR, V> {
  static __device__ __forceinline__ void run(V* v) {
    V a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    V c = cadd(v[1], v[3]), d = cmuli<DIR>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[1] = cadd(b, d);
    v[2] = csub(a, c);
    v[3] = csub(b, d);
  }
};

template <int DIR, typename V> struct Dft<5, DIR, V> {
  static __device__ __forceinline__ void run(V* v) {
    using T = typename Real<V>::type;
    V a1 = cadd(v[1], v[4]), a2 = cadd(v[2], v[3]);
    V b1 = csub(v[1], v[4]), b2 = csub(v[2], v[3]);
    V x1 = cadd(v[0], cadd(cscale(a1, (T)HPSI_C5_1), cscale(a2, (T)HPSI_C5_2)));
    V x2 = cadd(v[0], cadd(cscale(a1, (T)HPSI_C5_2), cscale(a2, (T)HPSI_C5_1)));
    V y1 = cmuli<DIR>(cadd(cscale(b1, (T)HPSI_S5_1), cscale(b2, (T)HPSI_S5_2)));
    V y2 = cmuli<DIR>(csub(cscale(b1, (T)HPSI_S5_2), cscale(b2, (T)HPSI_S5_1)));
    v[0] = cadd(v[0], cadd(a1, a2));
    v[1] = cadd(x1, y1);
    v[4] = csub(x1, y1);
    v[2] = cadd(x2, y2);
    v[3] = csub(x2, y2);
  }
};

template <typename V> __device__ __forceinline__ const V* tw_table(const FftPlan& p);
template <> __device__ __forceinline__ const double2* tw_table<double2>(const FftPlan& p) { return p.tw64; }
template <> __device__ __forceinline__ const float2* tw_table<float2>(const FftPlan& p) { return p.tw32; }

template <int R, int DIR, typename V>
__device__ __forceinline__ void warp_pass(V* line, int n, int Ns, const V* __restrict__ tw, int lane) {
  constexpr int MAXB = (kMaxFftN / R + 31) / 32;
  const int nbf = n / R;
  V v[MAXB][R];
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    const int j = lane + 32 * b;
    if (j < nbf) {
      const int kk = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = line[j + r * nbf];
#pragma unroll
      for (int r = 1; r < R; ++r) {
        V w = __ldg(tw + kk * (R - 1) + (r - 1));
        if (DIR > 0) w.y = -w.y;
        v[b][r] = cmul(v[b][r], w);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    const int j = lane + 32 * b;
    if (j < nbf) {
      Dft<R, DIR, V>::run(v[b]);
      const int kk = j % Ns;
      const int base = (j / Ns) * Ns * R + kk;
#pragma unroll
      for (int r = 0; r < R; ++r) line[base + r * Ns] = v[b][r];
    }
  }
  __syncwarp();
}

// Transform one line of length plan.n in shared memory; every lane of the warp must call it.
template <int DIR, typename V>
__device__ __forceinline__ void warp_fft(V* line, const FftPlan& plan, int lane) {
  const V* tw = tw_table<V>(plan);
  int Ns = 1;
  for (int s = 0; s < plan.nstages; ++s) {
    const int R = plan.radix[s];
    const V* t = tw + plan.twoff[s];
    if (R == 4) warp_pass<4, DIR>(line, plan.n, Ns, t, lane);
    else if (R == 2) warp_pass<2, DIR>(line, plan.n, Ns, t, lane);
    else if (R == 3) warp_pass<3, DIR>(line, plan.n, Ns, t, lane);
    else warp_pass<5, DIR>(line, plan.n, Ns, t, lane);
    Ns *= R;
  }
}

}  // namespace hpsi
