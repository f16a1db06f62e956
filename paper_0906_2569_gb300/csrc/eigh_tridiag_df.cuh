// Householder reduction of a real symmetric matrix to tridiagonal form in double-float arithmetic:
// every element of the trailing block, and every per-column scalar, is a pair of floats (hi, lo)
// whose sum carries ~48 significant bits, computed on the float32 pipes through error-free
// transformations (Knuth's TwoSum, Dekker's FastTwoSum, the FMA split of a product) and Newton steps
// from float32 seeds for 1/sqrt and 1/x.  On GB300 an SM issues float32 at 128 lanes per cycle and
// float64 at ~1.7, and a float64 instruction holds its scheduler's unit for ~64 cycles; the float64
// reduction (k_eh_tridiag_r) spends most of each column on serial float64 chains.  Here no float64
// instruction is left on a column's critical path: the float64 outputs (d, e, tau, the reflector
// scales) are written after the CTA has arrived at the grid barrier.
//
// Algorithm and data flow as k_eh_tridiag_r (eigh_tridiag_real.cuh): one pass over the own rows per
// column applies column j-1's rank-2 update and forms column j's matrix-vector product; one grid
// barrier per column publishes y, the CTAs' parts of s = v^T y (one pair per CTA, summed by every
// CTA after the barrier instead of float64 atomics) and the next row with its coefficients.  The
// reflector rows (vref) are stored as pairs; k_eh_vscale_df widens and scales them.  Relative
// accuracy ~1e-14 of the matrix norm (tests/test_gpu_eigh_real.py).  Included once, by eigh.cu,
// after eigh_tridiag_real.cuh.
#pragma once

#include <cuda_runtime.h>

#include "hpsi_internal.h"

namespace hpsi {
namespace {

// ---- double-float numbers: value x + y of a float2, |y| <= ulp(x) / 2 ----
// The _rn intrinsics are never contracted into FMAs or reassociated by the compiler.
__device__ __forceinline__ float2 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ float2 df_fast_sum(float a, float b) {   // exact when |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 df_of(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_val(float2 a) { return (double)a.x + (double)a.y; }
// a b = p + e: p = fl(a.x b.x), e the rest to float accuracy (a.y b.y dropped, ~2^-48 relative)
__device__ __forceinline__ void df_prod(float2 a, float2 b, float& p, float& e) {
  p = __fmul_rn(a.x, b.x);
  e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float2 s = df_two_sum(a.x, b.x);
  return df_fast_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  float p, e;
  df_prod(a, b, p, e);
  return df_fast_sum(p, e);
}
// acc + a u
__device__ __forceinline__ float2 df_mac(float2 acc, float2 a, float2 u) {
  float p, e;
  df_prod(a, u, p, e);
  const float2 s = df_two_sum(acc.x, p);
  return df_fast_sum(s.x, __fadd_rn(s.y, __fadd_rn(acc.y, e)));
}
// a - P u - Q y
__device__ __forceinline__ float2 df_rank2(float2 a, float2 P, float2 u, float2 Q, float2 y) {
  float p1, e1, p2, e2;
  df_prod(P, u, p1, e1);
  df_prod(Q, y, p2, e2);
  const float2 s1 = df_two_sum(a.x, -p1);
  const float2 s2 = df_two_sum(s1.x, -p2);
  const float lo = __fadd_rn(__fsub_rn(__fsub_rn(a.y, e1), e2), __fadd_rn(s1.y, s2.y));
  return df_fast_sum(s2.x, lo);
}
// 1 / sqrt(s) for s > 0: float32 seed, two Newton steps y += y (1 - s y^2) / 2 in pairs
__device__ __forceinline__ float2 df_rsqrt(float2 s) {
  float2 y = make_float2(rsqrtf(s.x), 0.f);
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float2 r = df_add(make_float2(1.f, 0.f), df_neg(df_mul(s, df_mul(y, y))));
    y = df_mac(y, df_mul(make_float2(0.5f, 0.f), y), r);
  }
  return y;
}
// 1 / d for d != 0: float32 seed, two Newton steps r += r (1 - d r) in pairs
__device__ __forceinline__ float2 df_rcp(float2 d) {
  float2 r = make_float2(__frcp_rn(d.x), 0.f);
#pragma unroll
  for (int it = 0; it < 2; ++it) r = df_mac(r, r, df_add(make_float2(1.f, 0.f), df_neg(df_mul(d, r))));
  return r;
}
__device__ __forceinline__ float2 df_shfl_xor(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ float2 df_warp_sum(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = df_add(v, df_shfl_xor(v, o));
  return v;
}

constexpr int kDfThreads = 512;                       // four warps per scheduler: the pairs' dependent
                                                      // chains need the extra warps to keep issuing
constexpr int kLoadKD = (kMaxNR + kDfThreads - 1) / kDfThreads;

__global__ void __launch_bounds__(kDfThreads, 1) k_eh_tridiag_df(TriArgsR p) {
  extern __shared__ double smd[];
  constexpr int NW = kDfThreads / 32;
  constexpr int kChainWarp = NW - 1;
  constexpr int kSumWarp = 2;      // sums the CTAs' parts of s after the barrier
  constexpr int kOutWarp = 3;      // writes the float64 outputs while the CTA waits at the barrier
  const int n = p.n, G = p.G, g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int R = g < n ? (n - 1 - g) / G + 1 : 0;
  const int Rmax = (n + G - 1) / G;
  // the float64 kernel's layout, every double slot holding one double-float pair
  float2* ubuf0 = reinterpret_cast<float2*>(smd);
  float2* ubuf1 = ubuf0 + n;
  float2* yP = ubuf0 + 2 * n;
  float2* rows = ubuf0 + 3 * n;
  float2* cA = rows + (size_t)Rmax * n;   // [Rmax] A_r, B_r, Q_r of the own rows
  float2* cB = cA + Rmax;
  float2* cQ = cB + Rmax;
  float2* pacc = cQ + Rmax;               // [4 Rmax] quarter (or whole-row) sums with u
  float2* pa1 = pacc + 4 * Rmax;          // [Rmax] element at column j+1 of each row
  float2* rnext = reinterpret_cast<float2*>(p.rnext);
  float2* ybuf = reinterpret_cast<float2*>(p.ybuf);
  float2* vref = reinterpret_cast<float2*>(p.vref);
  float2* rc2 = reinterpret_cast<float2*>(p.rowcoef);   // [2][4] A, B, Q, E of the published row
  float2* sp2 = reinterpret_cast<float2*>(p.spart);     // [2][G] each CTA's part of s
  __shared__ float2 red[NW];
  __shared__ float2 alpha_sh, dj_sh, tau_sh, scale_sh, beta_sh, ts_sh, hh_sh, pj_sh, qj_sh, ej_sh;
  const float2 zero2 = make_float2(0.f, 0.f), one2 = make_float2(1.f, 0.f);

  for (int lr = 0; lr < R; ++lr) {
    const int r = g + lr * G;
    for (int c = tid; c < n; c += kDfThreads) rows[(size_t)lr * n + c] = df_of(sym_at(p.a, p.lda, r, c));
  }
  float2 tau2 = zero2;     // tau_{j-1}^2
  int first = 0;           // the own rows r > j are lr = first .. R-1
  int jmodG = 0;           // j mod G: this CTA owns row j when jmodG == g
  for (int j = 0; j < n; ++j, jmodG = jmodG + 1 == G ? 0 : jmodG + 1) {
    if (first < R && g + first * G <= j) ++first;
    const int Ra = R - first;
    float2* uC = (j & 1) ? ubuf1 : ubuf0;   // this column's reflector, unscaled
    float2* uP = (j & 1) ? ubuf0 : ubuf1;   // previous column's
    // (A) row j and y of column j-1 into shared memory; one warp sums s_{j-1} and forms hh and row
    //     j's coefficients
    {
      float2 ra[kLoadKD], ya[kLoadKD];
#pragma unroll
      for (int k = 0; k < kLoadKD; ++k) {
        const int c = j + tid + k * kDfThreads;
        if (c < n) {
          if (j == 0) {
            ra[k] = df_of(sym_at(p.a, p.lda, 0, c));
          } else {
            ra[k] = __ldcg(rnext + ((j - 1) & 1) * n + c);
            ya[k] = __ldcg(ybuf + ((j - 1) & 1) * n + c);
          }
        }
      }
      if (wid == kSumWarp) {
        float2 hh = zero2, P = zero2, Q = zero2, E = zero2;
        if (j > 0) {
          const float2* sp = sp2 + ((j - 1) & 1) * G;
          float2 s = zero2;
          for (int q = lane; q < G; q += 32) s = df_add(s, __ldcg(sp + q));
          s = df_warp_sum(s);
          const float2* rc = rc2 + ((j - 1) & 1) * 4;
          hh = df_mul(make_float2(0.5f, 0.f), df_mul(tau2, s));
          P = df_rank2(__ldcg(rc), hh, __ldcg(rc + 1), zero2, zero2);   // A - hh B
          Q = __ldcg(rc + 2);
          E = __ldcg(rc + 3);
        }
        if (lane == 0) {
          hh_sh = hh;
          pj_sh = P;
          qj_sh = Q;
          ej_sh = E;
        }
      }
#pragma unroll
      for (int k = 0; k < kLoadKD; ++k) {
        const int c = j + tid + k * kDfThreads;
        if (c < n) {
          uC[c] = ra[k];
          if (j > 0) yP[c] = ya[k];
        }
      }
    }
    __syncthreads();
    // (B) column j-1's update of row j, its diagonal (thread 0: c = j), the reflector's vector uC[c]
    //     (c > j; thread 1 holds alpha at c = j+1) and sigma, two columns per step
    {
      const float2 Pj = pj_sh, Qj = qj_sh;
      float2 sg0 = zero2, sg1 = zero2;
      for (int c = j + tid; c < n; c += 2 * kDfThreads) {
        const int c2 = c + kDfThreads;
        float2 a = uC[c];
        float2 b = c2 < n ? uC[c2] : zero2;
        if (j > 0) {
          a = df_rank2(a, Pj, uP[c], Qj, yP[c]);
          if (c2 < n) b = df_rank2(b, Pj, uP[c2], Qj, yP[c2]);
        }
        if (c == j) {
          // the diagonal took its update in the published row but for E - 2 hh
          dj_sh = df_add(uC[c], df_neg(df_add(ej_sh, df_mul(make_float2(-2.f, 0.f), hh_sh))));
        } else {
          uC[c] = a;
          if (c == j + 1) alpha_sh = a;
          else sg0 = df_mac(sg0, a, a);
        }
        if (c2 < n) {
          uC[c2] = b;
          sg1 = df_mac(sg1, b, b);
        }
      }
      sg0 = df_warp_sum(df_add(sg0, sg1));
      if (lane == 0) red[wid] = sg0;
    }
    if (j == n - 1) {
      __syncthreads();
      if (g == 0 && tid == 0) p.d[j] = df_val(dj_sh);
      break;
    }
    __syncthreads();
    // (C) the chain warp: beta, tau, scale of column j in pairs;  all warps: own rows r > j
    if (wid == kChainWarp) {
      float2 sg = lane < NW ? red[lane] : zero2;
#pragma unroll
      for (int o = NW / 2; o > 0; o >>= 1) sg = df_add(sg, df_shfl_xor(sg, o));
      if (lane == 0) {
        const float2 ar = alpha_sh;
        float2 beta, tau, scale;
        if (sg.x == 0.f) {
          beta = ar;
          tau = zero2;
          scale = zero2;
        } else {
          const float2 S = df_mac(sg, ar, ar);
          const float2 y = df_rsqrt(S);
          const bool neg = __float_as_int(ar.x) < 0;            // beta = -sign(ar) |x|
          const float2 sy = df_mul(S, y);
          beta = neg ? sy : df_neg(sy);
          const float2 ib = neg ? y : df_neg(y);                 // 1 / beta
          tau = df_mac(one2, df_neg(ar), ib);                    // 1 - alpha / beta
          scale = df_rcp(df_add(ar, df_neg(beta)));              // 1 / (alpha - beta)
        }
        tau_sh = tau;
        scale_sh = scale;
        beta_sh = beta;
        ts_sh = df_mul(tau, scale);
      }
    }
    if (Ra > 0) {
      // every own row cut into quarters, the quarters round-robin over all warps; slot k of a row's
      // partial sums is its quarter k.  Two columns per lane and step (measured faster than four).
      const int m = n - 1 - j;
      const int quarter = split_chunk(m, 4);
      const float2 hhd = hh_sh;
      for (int it = wid; it < 4 * Ra; it += NW) {
        const int i = it >> 2, k = it & 3;
        const int c0 = j + 1 + k * quarter, c1 = min(n, c0 + quarter);
        const int lr = first + i;
        const int r = g + lr * G;
        float2* row = rows + (size_t)lr * n;
        const float2 P = df_rank2(cA[lr], hhd, cB[lr], zero2, zero2);   // A_r - hh B_r
        const float2 Q = cQ[lr];
        float2 ax = zero2, bx = zero2, a1 = zero2;
        for (int c = c0 + lane; c < c1; c += 64) {
          const int c2 = c + 32;
          const bool two = c2 < c1;
          float2 a = row[c];
          float2 b = two ? row[c2] : zero2;
          if (j > 0) {
            a = df_rank2(a, P, uP[c], Q, yP[c]);
            row[c] = a;
            if (two) {
              b = df_rank2(b, P, uP[c2], Q, yP[c2]);
              row[c2] = b;
            }
          }
          if (c == j + 1) a1 = a;
          else ax = df_mac(ax, a, uC[c]);
          if (two) bx = df_mac(bx, b, uC[c2]);
          if (r == j + 1) {
            rnext[(j & 1) * n + c] = a;
            if (two) rnext[(j & 1) * n + c2] = b;
          }
        }
        ax = df_warp_sum(df_add(ax, bx));
        if (lane == 0) {
          pacc[i * 4 + k] = ax;
          if (k == 0) pa1[i] = a1;
        }
      }
    }
    __syncthreads();
    // (D) warp 0: y_j[r] = a1 + scale * sum for the own rows and the CTA's part of s_j = v_j^T y_j;
    //     warp 1: row j+1's coefficients (and E = 2 tau y), published with it;
    //     the owner of row j stores u_j
    const float2 tauC = tau_sh, scC = scale_sh, tsC = ts_sh;
    auto row_y = [&](int i) {
      const float2 acc = df_add(df_add(pacc[i * 4], pacc[i * 4 + 1]), df_add(pacc[i * 4 + 2], pacc[i * 4 + 3]));
      return df_mac(pa1[i], scC, acc);
    };
    if (wid == 0) {
      float2 spd = zero2;
      for (int i = lane; i < Ra; i += 32) {
        const int r = g + (first + i) * G;
        const float2 y = row_y(i);
        ybuf[(j & 1) * n + r] = y;
        const float2 v = r == j + 1 ? one2 : df_mul(uC[r], scC);
        spd = df_mac(spd, v, y);
      }
      spd = df_warp_sum(spd);
      if (lane == 0) sp2[(j & 1) * G + g] = spd;
    } else if (wid == 1 && Ra > 0 && g + first * G == j + 1 && lane == 0) {
      // this CTA owns row j+1 (v = 1): A = tau scale y, B = 2 scale, Q = tau, E = 2 tau y
      const float2 y = row_y(0);
      float2* rc = rc2 + (j & 1) * 4;
      rc[0] = df_mul(tsC, y);
      rc[1] = df_mul(make_float2(2.f, 0.f), scC);
      rc[2] = tauC;
      rc[3] = df_mul(make_float2(2.f, 0.f), df_mul(tauC, y));
    }
    if (jmodG == g) {   // the owner of row j stores u_j (pairs; k_eh_vscale_df scales them)
      for (int c = j + 2 + tid; c < n; c += kDfThreads) vref[(size_t)j * n + c] = uC[c];
    }
    grid_arrive(p.bar);
    // while the other CTAs arrive: the own rows' coefficients for column j+1, tau_j^2, and (CTA 0)
    // the float64 outputs of column j
    if (wid == 1) {
      for (int i = lane; i < Ra; i += 32) {
        const int lr = first + i, r = g + lr * G;
        const float2 y = row_y(i);
        const float2 v = r == j + 1 ? one2 : df_mul(uC[r], scC);
        cA[lr] = df_mul(tsC, y);
        cB[lr] = df_mul(make_float2(2.f, 0.f), df_mul(scC, v));
        cQ[lr] = df_mul(tauC, v);
      }
    } else if (wid == kOutWarp && g == 0 && lane == 0) {
      const double be = df_val(beta_sh);
      p.d[j] = df_val(dj_sh);
      p.e[j] = be;
      p.e2[j] = be * be;
      p.tau[j] = df_val(tauC);
      p.vscale[j] = df_val(scC);
    }
    tau2 = df_mul(tauC, tauC);
    if (!grid_wait(p.bar, (unsigned)(G * (j + 1)), p.err)) return;
  }
}

// v_j[c] = u_j[c] scale_j for c > j + 1 (u_j stored as double-float pairs, turned into float64 in
// place) and v_j[j + 1] = 1.
__global__ void k_eh_vscale_df(int n, const double* __restrict__ vscale, double* __restrict__ vref) {
  const int j = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n - 1 || c <= j || c >= n) return;
  double* v = vref + (size_t)j * n + c;
  *v = c == j + 1 ? 1.0 : df_val(*reinterpret_cast<const float2*>(v)) * vscale[j];
}

}  // namespace
}  // namespace hpsi
