// Householder reduction of a dense real symmetric matrix to tridiagonal form: the first step of the
// reduced eigensolver of the Gamma-point Davidson (the reduced matrices of real orbitals are real
// symmetric).  The same scheme as the complex reduction in eigh_tridiag.cuh, in real arithmetic: a
// quarter of the float64 work per element and half the shared memory per row, so rows of up to
// 1824 columns fit on 152 SMs.  Included once, by eigh.cu, after eigh_tridiag.cuh (whose helpers it uses).
//
// Column j: x = A[j+1:, j] (row j of the symmetric matrix, updated), alpha = x_0,
// beta = -sign(alpha) |x|, tau = (beta - alpha) / beta, v = (x - beta e_1) / (alpha - beta) (so v_0 = 1,
// v_c = u_c scale for c > j+1 with u the updated row j and scale = 1 / (alpha - beta)); then with
// y = A22 v, s = v^T y, hh = tau^2 s / 2 the trailing block loses w v^T + v w^T, w = tau y - hh v.
// Element (r, c), c > j+1: a -= P_r u_c + Q_r y_c with P_r = A_r - hh B_r, A_r = tau scale y_r,
// B_r = 2 scale v_r, Q_r = tau v_r; the diagonal of row j+1 loses E - 2 hh with E = 2 tau y_{j+1}.
// As in the complex kernel, that update is applied to each row during the next column's pass over
// it, so every row is read and written once per column, and one grid barrier per column publishes
// y, s and the next row.
#pragma once

#include <cuda_runtime.h>

#include "hpsi_internal.h"

namespace hpsi {
namespace {

constexpr int kMaxNR = 2048;                          // largest n of the real reduction
constexpr int kLoadKR = (kMaxNR + 255) / 256;         // row elements per thread of the column loads

__device__ __forceinline__ double sym_at(const double* __restrict__ a, int lda, int r, int c) {
  return r <= c ? a[r + (size_t)c * lda] : a[c + (size_t)r * lda];
}

struct TriArgsR {
  int n, lda, G;
  const double* a;      // column-major, upper triangle read
  double* d;            // [n] diagonal of T
  double* e;            // [n] off-diagonal (e[j] couples j and j+1)
  double* e2;           // [n] e^2
  double* tau;          // [n] reflector factors
  double* vref;         // [n][n] row j: u_j at columns j+2..n-1
  double* ybuf;         // [2][n] y of the last two columns
  double* rnext;        // [2][n] the next row, published by its owner
  double* rowcoef;      // [2][4] coefficients of the published row: A, B, Q, E
  double* vscale;       // [n] scale of each reflector
  double* sacc;         // [4] s of the last columns (slot j & 3), accumulated by atomics
  unsigned int* bar;    // barrier arrival counter (zero at launch)
  int* err;             // device error word
  double* spart;        // [2][G] each CTA's part of s (the double-float kernel's pairs)
};

__global__ void __launch_bounds__(kTriThreads, 1) k_eh_tridiag_r(TriArgsR p) {
  extern __shared__ double smr[];
  constexpr int NW = kTriThreads / 32;
  constexpr int kChainWarp = NW - 1;
  const int n = p.n, G = p.G, g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int R = g < n ? (n - 1 - g) / G + 1 : 0;
  const int Rmax = (n + G - 1) / G;
  double* ubuf0 = smr;
  double* ubuf1 = smr + n;
  double* yP = smr + 2 * n;
  double* rows = smr + 3 * n;
  double* cA = rows + (size_t)Rmax * n;   // [Rmax] A_r, B_r, Q_r of the own rows
  double* cB = cA + Rmax;
  double* cQ = cB + Rmax;
  double* pacc = cQ + Rmax;               // [4 Rmax] quarter (or whole-row) sums with u
  double* pa1 = pacc + 4 * Rmax;          // [Rmax] element at column j+1 of each row
  __shared__ double red[NW];
  __shared__ double alpha_sh, tau_sh, scale_sh, beta_sh;

  for (int lr = 0; lr < R; ++lr) {
    const int r = g + lr * G;
    for (int c = tid; c < n; c += kTriThreads) rows[(size_t)lr * n + c] = sym_at(p.a, p.lda, r, c);
  }
  double tauPrev2 = 0.0;   // tau_{j-1}^2
  int first = 0;           // the own rows r > j are lr = first .. R-1
  int jmodG = 0;           // j mod G: this CTA owns row j when jmodG == g
  for (int j = 0; j < n; ++j, jmodG = jmodG + 1 == G ? 0 : jmodG + 1) {
    if (first < R && g + first * G <= j) ++first;
    const int Ra = R - first;
    double* uC = (j & 1) ? ubuf1 : ubuf0;   // this column's reflector, unscaled
    double* uP = (j & 1) ? ubuf0 : ubuf1;   // previous column's
    // (A) row j and y of column j-1 into shared memory; s, hh and row j's coefficients
    double hh = 0.0, Pj = 0.0, Qj = 0.0, Ej = 0.0;
    {
      double sv = 0.0, A = 0.0, B = 0.0;
      if (j > 0) {
        const double* rc = p.rowcoef + ((j - 1) & 1) * 4;
        sv = __ldcg(&p.sacc[(j - 1) & 3]);
        A = __ldcg(&rc[0]);
        B = __ldcg(&rc[1]);
        Qj = __ldcg(&rc[2]);
        Ej = __ldcg(&rc[3]);
      }
      double ra[kLoadKR], ya[kLoadKR];
#pragma unroll
      for (int k = 0; k < kLoadKR; ++k) {
        const int c = j + tid + k * kTriThreads;
        if (c < n) {
          if (j == 0) {
            ra[k] = sym_at(p.a, p.lda, 0, c);
          } else {
            ra[k] = __ldcg(&p.rnext[((j - 1) & 1) * n + c]);
            ya[k] = __ldcg(&p.ybuf[((j - 1) & 1) * n + c]);
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
      if (j > 0) {
        hh = 0.5 * tauPrev2 * sv;
        Pj = fma(-hh, B, A);
      }
    }
    if (g == 0 && tid == 0) p.sacc[(j + 2) & 3] = 0.0;   // slot of column j-2, read at the start of j-1
    __syncthreads();
    // (B) column j-1's update of row j, its diagonal, the reflector's vector uC[c] (c > j) and sigma
    double sig = 0.0, dj = 0.0;
    for (int c = j + tid; c < n; c += kTriThreads) {
      double a = uC[c];
      if (c == j) {
        dj = a - (Ej - 2.0 * hh);
      } else {
        if (j > 0) a = fma(-Pj, uP[c], fma(-Qj, yP[c], a));
        uC[c] = a;
        if (c == j + 1) alpha_sh = a;
        else sig = fma(a, a, sig);
      }
    }
    if (j == n - 1) {
      if (g == 0 && tid == 0) p.d[j] = dj;
      break;
    }
    sig = warp_sum(sig);
    if (lane == 0) red[wid] = sig;
    __syncthreads();
    // (C) the chain warp: beta, tau, scale of column j;  all warps: own rows r > j, in parts
    if (wid == kChainWarp) {
      double sg = lane < NW ? red[lane] : 0.0;
      sg += __shfl_xor_sync(0xffffffffu, sg, 4);
      sg += __shfl_xor_sync(0xffffffffu, sg, 2);
      sg += __shfl_xor_sync(0xffffffffu, sg, 1);
      if (lane == 0) {
        const double ar = alpha_sh;
        double beta, tau, scale;
        if ((__double_as_longlong(sg) << 1) == 0) {
          beta = ar;
          tau = 0.0;
          scale = 0.0;
        } else {
          const double S = fma(ar, ar, sg);
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
      // complex reduction); slot k of a row's partial sums is its quarter k
      const int m = n - 1 - j;
      const int rem = Ra & 3, full = Ra - rem;
      const int sched = wid & 3, half = wid >> 2;
      const int quarter = split_chunk(m, 4);
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
        double* row = rows + (size_t)lr * n;
        const double P = fma(-hh, cB[lr], cA[lr]);
        const double Q = cQ[lr];
        double ax = 0.0, bx = 0.0, a1 = 0.0;
        for (int c = c0 + lane; c < c1; c += 64) {
          const int c2 = c + 32;
          const bool two = c2 < c1;
          double a = row[c];
          double b = two ? row[c2] : 0.0;
          if (j > 0) {
            a = fma(-P, uP[c], fma(-Q, yP[c], a));
            row[c] = a;
            if (two) {
              b = fma(-P, uP[c2], fma(-Q, yP[c2], b));
              row[c2] = b;
            }
          }
          if (c == j + 1) a1 = a;
          else ax = fma(a, uC[c], ax);
          if (two) bx = fma(b, uC[c2], bx);
          if (r == j + 1) {
            p.rnext[(j & 1) * n + c] = a;
            if (two) p.rnext[(j & 1) * n + c2] = b;
          }
        }
        ax = warp_sum(ax + bx);
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
      double acc = pacc[i * 4];
      if (i >= Ra - (Ra & 3)) acc += (pacc[i * 4 + 1] + pacc[i * 4 + 2]) + pacc[i * 4 + 3];
      return fma(scC, acc, pa1[i]);
    };
    auto coefs = [&](int r, double y, double* A, double* B, double* Q) {
      const double v = r == j + 1 ? 1.0 : uC[r] * scC;
      *A = tauC * scC * y;
      *B = 2.0 * scC * v;
      *Q = tauC * v;
    };
    if (wid == 0) {
      double sp = 0.0;
      for (int i = lane; i < Ra; i += 32) {
        const int r = g + (first + i) * G;
        const double y = row_y(i);
        p.ybuf[(j & 1) * n + r] = y;
        sp = fma(r == j + 1 ? 1.0 : uC[r] * scC, y, sp);
      }
      sp = warp_sum(sp);
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
    if (jmodG == g) {   // the owner of row j stores u_j; the back-transformation scales it
      for (int c = j + 2 + tid; c < n; c += kTriThreads) p.vref[(size_t)j * n + c] = uC[c];
    }
    grid_arrive(p.bar);
    if (wid == 1) {
      for (int i = lane; i < Ra; i += 32) {
        const int lr = first + i, r = g + lr * G;
        double A, B, Q;
        coefs(r, row_y(i), &A, &B, &Q);
        cA[lr] = A;
        cB[lr] = B;
        cQ[lr] = Q;
      }
    }
    tauPrev2 = tauC * tauC;
    if (!grid_wait(p.bar, (unsigned)(G * (j + 1)), p.err)) return;
  }
}

}  // namespace
}  // namespace hpsi
