// Householder reduction of a real symmetric matrix to tridiagonal form with the row work in
// double-float arithmetic: every element of the trailing block is a pair of floats (hi, lo) whose
// sum carries ~48 significant bits, and the per-column rank-2 update and dot product run on the
// float32 pipes through error-free transformations (Knuth's TwoSum, Dekker's FastTwoSum and the
// FMA split of a product).  On GB300 an SM issues float32 at 128 lanes per cycle against ~1.7 for
// float64, so ~40 float32 operations per element still beat the 3 float64 FMAs of the float64
// kernel several times over.  The scalars of each column (the reflector's beta, tau and scale, the
// rows' coefficients, s and the diagonal) stay float64.
//
// Same algorithm and data flow as k_eh_tridiag_r (eigh_tridiag_real.cuh): one pass over the own
// rows per column that applies column j-1's rank-2 update and forms column j's matrix-vector
// product, one grid barrier per column.  The published row, y and the reflector rows (vref) are
// double-float pairs; k_eh_vscale_df turns the reflector rows into float64 afterwards.  Relative
// accuracy ~1e-13 of the matrix norm: for reduced problems whose eigenvectors rotate a float32
// basis.  Included once, by eigh.cu, after eigh_tridiag_real.cuh.
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
__device__ __forceinline__ float2 df_warp_sum(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float2 w;
    w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    v = df_add(v, w);
  }
  return v;
}

__global__ void __launch_bounds__(kTriThreads, 1) k_eh_tridiag_df(TriArgsR p) {
  extern __shared__ double smd[];
  constexpr int NW = kTriThreads / 32;
  constexpr int kChainWarp = NW - 1;
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
  __shared__ float2 red[NW];
  __shared__ double alpha_sh, tau_sh, scale_sh, beta_sh, hh_sh, ej_sh;
  __shared__ float2 pj_sh, qj_sh, hhd_sh;

  for (int lr = 0; lr < R; ++lr) {
    const int r = g + lr * G;
    for (int c = tid; c < n; c += kTriThreads) rows[(size_t)lr * n + c] = df_of(sym_at(p.a, p.lda, r, c));
  }
  double tauPrev2 = 0.0;   // tau_{j-1}^2
  int first = 0;           // the own rows r > j are lr = first .. R-1
  int jmodG = 0;           // j mod G: this CTA owns row j when jmodG == g
  for (int j = 0; j < n; ++j, jmodG = jmodG + 1 == G ? 0 : jmodG + 1) {
    if (first < R && g + first * G <= j) ++first;
    const int Ra = R - first;
    float2* uC = (j & 1) ? ubuf1 : ubuf0;   // this column's reflector, unscaled
    float2* uP = (j & 1) ? ubuf0 : ubuf1;   // previous column's
    // (A) row j and y of column j-1 into shared memory; s, hh and row j's coefficients (one lane)
    {
      float2 ra[kLoadKR], ya[kLoadKR];
#pragma unroll
      for (int k = 0; k < kLoadKR; ++k) {
        const int c = j + tid + k * kTriThreads;
        if (c < n) {
          if (j == 0) {
            ra[k] = df_of(sym_at(p.a, p.lda, 0, c));
          } else {
            const float2* rs = rnext + ((j - 1) & 1) * n + c;
            const float2* ys = ybuf + ((j - 1) & 1) * n + c;
            ra[k] = __ldcg(rs);
            ya[k] = __ldcg(ys);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kLoadKR; ++k) {
        const int c = j + tid + k * kTriThreads;
        if (c < n) {
          uC[c] = ra[k];
          if (j > 0) yP[c] = ya[k];
        }
      }
      if (tid == 0) {
        double hh = 0.0, Pj = 0.0, Qj = 0.0, Ej = 0.0;
        if (j > 0) {
          const double* rc = p.rowcoef + ((j - 1) & 1) * 4;
          const double sv = __ldcg(&p.sacc[(j - 1) & 3]);
          hh = 0.5 * tauPrev2 * sv;
          Pj = fma(-hh, __ldcg(&rc[1]), __ldcg(&rc[0]));
          Qj = __ldcg(&rc[2]);
          Ej = __ldcg(&rc[3]);
        }
        hh_sh = hh;
        ej_sh = Ej;
        pj_sh = df_of(Pj);
        qj_sh = df_of(Qj);
        hhd_sh = df_of(hh);
      }
    }
    if (g == 0 && tid == 0) p.sacc[(j + 2) & 3] = 0.0;   // slot of column j-2, read at the start of j-1
    __syncthreads();
    const double hh = hh_sh;
    // (B) column j-1's update of row j, its diagonal, the reflector's vector uC[c] (c > j) and sigma
    float2 sig = make_float2(0.f, 0.f);
    double dj = 0.0;
    {
      const float2 Pj = pj_sh, Qj = qj_sh;
      for (int c = j + tid; c < n; c += kTriThreads) {
        float2 a = uC[c];
        if (c == j) {
          dj = df_val(a) - (ej_sh - 2.0 * hh);
        } else {
          if (j > 0) a = df_rank2(a, Pj, uP[c], Qj, yP[c]);
          uC[c] = a;
          if (c == j + 1) alpha_sh = df_val(a);
          else sig = df_mac(sig, a, a);
        }
      }
    }
    if (j == n - 1) {
      if (g == 0 && tid == 0) p.d[j] = dj;
      break;
    }
    sig = df_warp_sum(sig);
    if (lane == 0) red[wid] = sig;
    __syncthreads();
    // (C) the chain warp: beta, tau, scale of column j;  all warps: own rows r > j, in parts
    if (wid == kChainWarp) {
      float2 sg = lane < NW ? red[lane] : make_float2(0.f, 0.f);
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        float2 w;
        w.x = __shfl_xor_sync(0xffffffffu, sg.x, o);
        w.y = __shfl_xor_sync(0xffffffffu, sg.y, o);
        sg = df_add(sg, w);
      }
      if (lane == 0) {
        const double ar = alpha_sh, sgd = df_val(sg);
        double beta, tau, scale;
        if ((__double_as_longlong(sgd) << 1) == 0) {
          beta = ar;
          tau = 0.0;
          scale = 0.0;
        } else {
          const double S = fma(ar, ar, sgd);
          const double y = rsqrt_nr(S);
          const bool neg = __double_as_longlong(ar) < 0;     // beta = -sign(ar) |x|
          beta = neg ? S * y : -(S * y);
          const double ib = neg ? y : -y;                    // 1 / beta
          tau = fma(-ar, ib, 1.0);
          scale = recip_nr(ar - beta);                       // 1 / (alpha - beta)
        }
        tau_sh = tau;
        scale_sh = scale;
        beta_sh = beta;
      }
    }
    if (Ra > 0) {
      // whole rows round-robin over the four schedulers, leftover rows cut into quarters (as in the
      // float64 kernel); slot k of a row's partial sums is its quarter k
      const int m = n - 1 - j;
      const int rem = Ra & 3, full = Ra - rem;
      const int sched = wid & 3, half = wid >> 2;
      const int quarter = split_chunk(m, 4);
      const float2 hhd = hhd_sh, zero2 = make_float2(0.f, 0.f);
      int ord = 0;
      for (int it = sched; it < full + 4 * rem; it += 4, ++ord) {
        if ((ord & 1) != half) continue;
        int i, k, c0, c1;
        if (it < full) {
          i = it;
          k = 0;
          c0 = j + 1;
          c1 = n;
        } else {
          i = full + (it - full) / 4;
          k = sched;
          c0 = j + 1 + k * quarter;
          c1 = min(n, c0 + quarter);
        }
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
    // (D) warp 0: y_j[r] = a1 + scale * sum for the own rows and their part of s_j = v_j^T y_j;
    //     warp 1: the own rows' A, B, Q for column j+1 (E for row j+1, published with it);
    //     the owner of row j stores u_j; CTA 0 the outputs of column j
    const double tauC = tau_sh, scC = scale_sh;
    auto row_y = [&](int i) {
      float2 acc = pacc[i * 4];
      if (i >= Ra - (Ra & 3)) acc = df_add(df_add(acc, pacc[i * 4 + 1]), df_add(pacc[i * 4 + 2], pacc[i * 4 + 3]));
      return fma(scC, df_val(acc), df_val(pa1[i]));
    };
    auto coefs = [&](int r, double y, double* A, double* B, double* Q) {
      const double v = r == j + 1 ? 1.0 : df_val(uC[r]) * scC;
      *A = tauC * scC * y;
      *B = 2.0 * scC * v;
      *Q = tauC * v;
    };
    if (wid == 0) {
      // y and s in double-float (float64 only for the scale and the final sum)
      const float2 scD = df_of(scC), one2 = make_float2(1.f, 0.f);
      float2 spd = make_float2(0.f, 0.f);
      for (int i = lane; i < Ra; i += 32) {
        const int r = g + (first + i) * G;
        float2 acc = pacc[i * 4];
        if (i >= Ra - (Ra & 3)) acc = df_add(df_add(acc, pacc[i * 4 + 1]), df_add(pacc[i * 4 + 2], pacc[i * 4 + 3]));
        const float2 y = df_mac(pa1[i], scD, acc);
        ybuf[(j & 1) * n + r] = y;
        float2 v = one2;
        if (r != j + 1) v = df_mac(make_float2(0.f, 0.f), uC[r], scD);
        spd = df_mac(spd, v, y);
      }
      const double sp = df_val(df_warp_sum(spd));
      if (lane == 0) {
        atomicAdd(&p.sacc[j & 3], sp);
        if (g == 0) {
          p.d[j] = dj;
          p.e[j] = beta_sh;
          p.e2[j] = beta_sh * beta_sh;
          p.tau[j] = tauC;
          p.vscale[j] = scC;
        }
      }
    } else if (wid == 1 && Ra > 0 && g + first * G == j + 1 && lane == 0) {
      // this CTA owns row j+1: publish its coefficients (and E = 2 tau y) before arriving
      const double y = row_y(0);
      double A, B, Q;
      coefs(j + 1, y, &A, &B, &Q);
      double* rc = p.rowcoef + (j & 1) * 4;
      rc[0] = A;
      rc[1] = B;
      rc[2] = Q;
      rc[3] = 2.0 * tauC * y;
    }
    if (jmodG == g) {   // the owner of row j stores u_j (pairs; k_eh_vscale_df scales them)
      for (int c = j + 2 + tid; c < n; c += kTriThreads) vref[(size_t)j * n + c] = uC[c];
    }
    grid_arrive(p.bar);
    if (wid == 1) {
      for (int i = lane; i < Ra; i += 32) {
        const int lr = first + i, r = g + lr * G;
        double A, B, Q;
        coefs(r, row_y(i), &A, &B, &Q);
        cA[lr] = df_of(A);
        cB[lr] = df_of(B);
        cQ[lr] = df_of(Q);
      }
    }
    tauPrev2 = tauC * tauC;
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
