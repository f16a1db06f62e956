// Householder reduction of a dense Hermitian matrix to real symmetric tridiagonal form: the first
// step of the reduced eigensolver in eigh.cu, kept in its own file so that its measured DRAM traffic
// can be keyed to the code that produces it.  Included once, by eigh.cu.
#pragma once

#include <cuda_runtime.h>

#include "hpsi_internal.h"

namespace hpsi {
namespace {

constexpr int kTriThreads = 256;                     // threads per CTA of the reduction
constexpr int kMaxN = 1024;                          // largest n handled here
constexpr int kLoadK = (kMaxN + 255) / 256;          // row elements per thread of the column loads
constexpr long long kBarrierLimit = 2000000000LL;    // clock cycles (about 1 s) per barrier wait

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a - w1 conj(v1) - v2 conj(w2) as eight fused multiply-adds
__device__ __forceinline__ double2 rank2_sub(double2 a, double2 w1, double2 v1, double2 v2, double2 w2) {
  double x = fma(-w1.x, v1.x, a.x);
  x = fma(-w1.y, v1.y, x);
  x = fma(-v2.x, w2.x, x);
  x = fma(-v2.y, w2.y, x);
  double y = fma(-w1.y, v1.x, a.y);
  y = fma(w1.x, v1.y, y);
  y = fma(-v2.y, w2.x, y);
  y = fma(v2.x, w2.y, y);
  return make_double2(x, y);
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Element (r, c) of the Hermitian matrix whose upper triangle is a (column-major, leading dim lda).
__device__ __forceinline__ double2 herm_at(const double2* __restrict__ a, int lda, int r, int c) {
  if (r <= c) {
    double2 v = a[r + (size_t)c * lda];
    if (r == c) v.y = 0.0;
    return v;
  }
  double2 v = a[c + (size_t)r * lda];
  v.y = -v.y;
  return v;
}

struct TriArgs {
  int n, lda, G;
  const double2* a;
  double* d;            // [n] diagonal of T
  double* e;            // [n] off-diagonal of T (e[j] couples j and j+1)
  double* e2;           // [n] e^2
  double2* tau;         // [n] reflector factors
  double2* vref;        // [n][n] row j: v_j at columns j+1..n-1
  double2* ybuf;        // [2][n] y of the last two columns
  double2* rnext;       // [2][n] the next row, published by its owner
  double2* rowcoef;     // [2][4] coefficients of the published row: A, B, Q, (E, 0)
  double2* vscale;      // [n] scale of each reflector
  double* sacc;         // [4] s of the last columns (slot j & 3), accumulated by atomics
  unsigned int* bar;    // barrier arrival counter (zero at launch)
  int* err;             // device error word
};

// Grid-wide barrier of a cooperative launch on a monotonic arrival counter: barrier number k
// (k = 1, 2, ...) is passed once the counter reaches k G.  Arrival (after a CTA barrier, so every
// thread's writes precede it) adds 1 with release semantics; the wait polls with acquire loads, so
// neither a reset nor a generation flip sits between the last arrival and the release.  The two are
// separate so that a CTA can do local work between them.  grid_wait returns false when this CTA's
// wait ran out or another CTA reported a failure (the error word is then set).
__device__ __forceinline__ void grid_arrive(unsigned int* count) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
}

__device__ bool grid_wait(unsigned int* count, unsigned int target, int* err) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    int good = 1;
    const long long t0 = clock64();
    unsigned int spins = 0;
    for (;;) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if ((int)(v - target) >= 0) break;
      if ((++spins & 255u) == 0u && (*(volatile int*)err != 0 || clock64() - t0 > kBarrierLimit)) {
        atomicCAS(err, 0, 3);
        good = 0;
        break;
      }
    }
    ok = good && *(volatile int*)err == 0;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ int biased_exp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }

// 1/x by two Newton-Raphson steps r <- r (2 - x r) from a float32 seed (quadratic convergence:
// 2^-23 -> 2^-46 -> 2^-92); plain division outside |x| in [2^-100, 2^100].  Four float64
// operations instead of the 600-cycle division sequence.
__device__ __forceinline__ double recip_nr(double x) {
  const int ex = biased_exp(x);
  if (ex < 1023 - 100 || ex > 1023 + 100) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// 1/sqrt(x) for x > 0 by two Newton steps y <- y (3/2 - (x/2) y^2) from a float32 seed; library
// sqrt and division outside x in [2^-100, 2^100].
__device__ __forceinline__ double rsqrt_nr(double x) {
  const int ex = biased_exp(x);
  if (ex < 1023 - 100 || ex > 1023 + 100) return 1.0 / sqrt(x);
  const double h = 0.5 * x;
  double y = (double)rsqrtf((float)x);
  y = y * fma(-h, y * y, 1.5);
  y = y * fma(-h, y * y, 1.5);
  return y;
}

// Column chunk of one of q parts of a row of m columns, rounded up to whole warps (no division).
__device__ __forceinline__ int split_chunk(int m, int q) {
  const int c = q == 1 ? m : q == 2 ? (m + 1) >> 1 : q == 4 ? (m + 3) >> 2 : ((m + 2) * 0x5556) >> 16;
  return (c + 31) & ~31;
}

__device__ __forceinline__ double2 cmulc2(double2 a, double2 b) {   // a * conj(b)
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

// Column j keeps the previous reflector in a folded form: with u the updated row j-1 (so
// v_{j-1}[c] = conj(u[c]) scale for c > j, v_{j-1}[j] = 1) and w = tau y - hh v (hh = |tau|^2 s / 2,
// s = v^H y), the rank-2 update of element (r, c), c > j, is
//   a -= P_r u[c] + Q_r conj(y[c]),  P_r = A_r - hh B_r,  A_r = tau y_r conj(scale),
//   B_r = 2 v_r conj(scale),  Q_r = conj(tau) v_r,
// and the diagonal element of row j loses E_j - 2 hh with E_j = 2 Re(tau y_j).  A, B, Q (and E)
// are formed for every row before the barrier; after it only hh is new.  The new reflector enters
// the product with A as conj(u) and its scale is applied to each row sum at the end, so one warp
// computes the reflector's scalars while the others update the rows.  s is accumulated across
// CTAs by float64 atomics.  The own rows' work is cut into parts spread over the eight warps
// (two per scheduler) so that each scheduler carries the same float64 work: a scheduler issues
// float64 at its own fixed rate, and a CTA barrier does not wait for float64 work still queued.
__global__ void __launch_bounds__(kTriThreads, 1) k_eh_tridiag(TriArgs p) {
  extern __shared__ double2 sm[];
  constexpr int NW = kTriThreads / 32;
  constexpr int kChainWarp = NW - 1;
  const int n = p.n, G = p.G, g = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int R = g < n ? (n - 1 - g) / G + 1 : 0;
  const int Rmax = (n + G - 1) / G;
  double2* ubuf0 = sm;
  double2* ubuf1 = sm + n;
  double2* yP = sm + 2 * n;
  double2* rows = sm + 3 * n;
  double2* cA = rows + (size_t)Rmax * n;   // [Rmax] A_r, B_r, Q_r of the own rows
  double2* cB = cA + Rmax;
  double2* cQ = cB + Rmax;
  double2* pacc = cQ + Rmax;               // [4 Rmax] quarter (or whole-row) sums with conj(u)
  double2* pa1 = pacc + 4 * Rmax;          // [Rmax] element at column j+1 of each row
  __shared__ double red[NW];
  __shared__ double2 alpha_sh, tau_sh, scale_sh, tcs_sh, cts_sh;
  __shared__ double beta_sh, s2_sh;

  for (int lr = 0; lr < R; ++lr) {
    const int r = g + lr * G;
    for (int c = tid; c < n; c += kTriThreads) rows[(size_t)lr * n + c] = herm_at(p.a, p.lda, r, c);
  }
  double2 scP = make_double2(0.0, 0.0);
  double tauAbs2 = 0.0;   // |tau_{j-1}|^2
  int first = 0;          // the own rows r > j are lr = first .. R-1
  int jmodG = 0;          // j mod G: this CTA owns row j when jmodG == g
  for (int j = 0; j < n; ++j, jmodG = jmodG + 1 == G ? 0 : jmodG + 1) {
    if (first < R && g + first * G <= j) ++first;   // j passed an own row (at most one per column)
    const int Ra = R - first;
    double2* uC = (j & 1) ? ubuf1 : ubuf0;   // this column's reflector, unscaled
    double2* uP = (j & 1) ? ubuf0 : ubuf1;   // previous column's
    // (A) row j and y of column j-1 into shared memory; s, hh and row j's coefficients (every load
    //     is issued before the first use)
    double hh = 0.0;
    double2 Pj = make_double2(0.0, 0.0), Qj = Pj;
    double Ej = 0.0;
    {
      double sv = 0.0;
      double2 A = Pj, B = Pj;
      if (j > 0) {
        const double2* rc = p.rowcoef + ((j - 1) & 1) * 4;
        sv = __ldcg(&p.sacc[(j - 1) & 3]);
        A = __ldcg(&rc[0]);
        B = __ldcg(&rc[1]);
        Qj = __ldcg(&rc[2]);
        Ej = __ldcg(&rc[3]).x;
      }
      double2 ra[kLoadK], ya[kLoadK];
#pragma unroll
      for (int k = 0; k < kLoadK; ++k) {
        const int c = j + tid + k * kTriThreads;
        if (c < n) {
          if (j == 0) {
            ra[k] = herm_at(p.a, p.lda, 0, c);
          } else {
            ra[k] = __ldcg(&p.rnext[((j - 1) & 1) * n + c]);
            ya[k] = __ldcg(&p.ybuf[((j - 1) & 1) * n + c]);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < kLoadK; ++k) {
        const int c = j + tid + k * kTriThreads;
        if (c < n) {
          uC[c] = ra[k];
          if (j > 0) yP[c] = ya[k];
        }
      }
      if (j > 0) {
        hh = 0.5 * tauAbs2 * sv;
        Pj = make_double2(fma(-hh, B.x, A.x), fma(-hh, B.y, A.y));
      }
    }
    if (g == 0 && tid == 0) p.sacc[(j + 2) & 3] = 0.0;   // slot of column j-2, read at the start of j-1
    __syncthreads();
    // (B) column j-1's update of row j, its diagonal, the reflector's vector uC[c] (c > j) and sigma
    double sig = 0.0, dj = 0.0;
    for (int c = j + tid; c < n; c += kTriThreads) {
      double2 a = uC[c];
      if (c == j) {
        dj = a.x - (Ej - 2.0 * hh);
      } else {
        if (j > 0) a = rank2_sub(a, Pj, make_double2(uP[c].x, -uP[c].y), Qj, yP[c]);
        uC[c] = a;
        if (c == j + 1) alpha_sh = make_double2(a.x, -a.y);
        else sig = fma(a.x, a.x, fma(a.y, a.y, sig));
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
        const double ar = alpha_sh.x, ai = alpha_sh.y;
        double beta;
        double2 tau, scale;
        if ((__double_as_longlong(sg) << 1) == 0 && (__double_as_longlong(ai) << 1) == 0) {
          beta = ar;
          tau = make_double2(0.0, 0.0);
          scale = make_double2(0.0, 0.0);
        } else {
          const double S = fma(ar, ar, fma(ai, ai, sg));
          const double y = rsqrt_nr(S);
          const bool neg = __double_as_longlong(ar) < 0;     // beta = -sign(ar) |x|
          beta = neg ? S * y : -(S * y);
          const double ib = neg ? y : -y;                    // 1 / beta
          tau = make_double2(fma(-ar, ib, 1.0), -ai * ib);
          const double dr = ar - beta;
          const double iden = recip_nr(fma(dr, dr, ai * ai));
          scale = make_double2(dr * iden, -ai * iden);       // 1 / (alpha - beta)
        }
        tau_sh = tau;
        scale_sh = scale;
        beta_sh = beta;
        tcs_sh = cmulc2(tau, scale);                                         // tau conj(scale)
        cts_sh = cmul(make_double2(tau.x, -tau.y), scale);                   // conj(tau) scale
        s2_sh = 2.0 * fma(scale.x, scale.x, scale.y * scale.y);              // 2 |scale|^2
      }
    }
    if (Ra > 0) {
      // whole rows go round-robin to the four schedulers (warp & 3), each leftover row is cut into
      // quarters, one per scheduler, so every scheduler carries Ra / 4 rows of float64 work; the two
      // warps of a scheduler (wid and wid + 4) alternate over its items.  Slot k of a row's partial
      // sums is its quarter k (slot 0 for a whole row, which then holds column j+1).
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
          i = full + (it - full) / 4;   // it - full = 4 t + sched
          k = sched;
          c0 = j + 1 + k * quarter;
          c1 = min(n, c0 + quarter);
        }
        const int lr = first + i;
        const int r = g + lr * G;
        double2* row = rows + (size_t)lr * n;
        const double2 P = make_double2(fma(-hh, cB[lr].x, cA[lr].x), fma(-hh, cB[lr].y, cA[lr].y));
        const double2 Q = cQ[lr];
        double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
        double2 a1 = make_double2(0.0, 0.0);
        for (int c = c0 + lane; c < c1; c += 64) {
          const int c2 = c + 32;
          const bool two = c2 < c1;
          double2 a = row[c];
          double2 b = two ? row[c2] : make_double2(0.0, 0.0);
          if (j > 0) {
            a = rank2_sub(a, P, make_double2(uP[c].x, -uP[c].y), Q, yP[c]);
            row[c] = a;
            if (two) {
              b = rank2_sub(b, P, make_double2(uP[c2].x, -uP[c2].y), Q, yP[c2]);
              row[c2] = b;
            }
          }
          if (c == j + 1) {
            a1 = a;
          } else {
            const double2 u = uC[c];            // a * conj(u)
            ax = fma(a.x, u.x, fma(a.y, u.y, ax));
            ay = fma(a.y, u.x, fma(-a.x, u.y, ay));
          }
          if (two) {
            const double2 u = uC[c2];
            bx = fma(b.x, u.x, fma(b.y, u.y, bx));
            by = fma(b.y, u.x, fma(-b.x, u.y, by));
          }
          if (r == j + 1) {
            p.rnext[(j & 1) * n + c] = a;
            if (two) p.rnext[(j & 1) * n + c2] = b;
          }
        }
        ax = warp_sum(ax + bx);
        ay = warp_sum(ay + by);
        if (lane == 0) {
          pacc[i * 4 + k] = make_double2(ax, ay);
          if (k == 0) pa1[i] = a1;
        }
      }
    }
    __syncthreads();
    // (D) warp 0: y_j[r] = a1 + scale * sum for the own rows and their part of s_j = v_j^H y_j;
    //     warp 1: the own rows' A, B, Q for column j+1 (and E for row j+1, published with it);
    //     the owner of row j stores v_j; CTA 0 the outputs of column j
    const double2 tauC = tau_sh, scC = scale_sh;
    const double2 cscC = make_double2(scC.x, -scC.y);
    const double2 tcs = tcs_sh, cts = cts_sh;
    const double s2 = s2_sh;
    // the own rows' y_j (lanes of warps 0 and 1 over the rows) and the coefficients of column j's
    // update for row lr: A = tau y conj(scale), B = 2 v conj(scale), Q = conj(tau) v
    auto row_y = [&](int i) {
      double2 acc = pacc[i * 4];
      if (i >= Ra - (Ra & 3)) {   // a leftover row: four quarters
        acc.x += (pacc[i * 4 + 1].x + pacc[i * 4 + 2].x) + pacc[i * 4 + 3].x;
        acc.y += (pacc[i * 4 + 1].y + pacc[i * 4 + 2].y) + pacc[i * 4 + 3].y;
      }
      const double2 a1 = pa1[i];
      return make_double2(fma(scC.x, acc.x, fma(-scC.y, acc.y, a1.x)), fma(scC.x, acc.y, fma(scC.y, acc.x, a1.y)));
    };
    auto coefs = [&](int lr, int r, double2 y, double2* A, double2* B, double2* Q) {
      const bool lead = r == j + 1;                       // v_j[j+1] = 1, else v_j[r] = conj(u_r) scale
      const double2 cu = make_double2(uC[r].x, -uC[r].y);
      *A = cmul(y, tcs);
      *B = lead ? make_double2(2.0 * scC.x, -2.0 * scC.y) : make_double2(s2 * cu.x, s2 * cu.y);
      *Q = lead ? make_double2(tauC.x, -tauC.y) : cmul(cu, cts);
    };
    if (wid == 0) {
      double sp = 0.0;
      for (int i = lane; i < Ra; i += 32) {
        const int r = g + (first + i) * G;
        const double2 y = row_y(i);
        p.ybuf[(j & 1) * n + r] = y;
        // Re(conj(v_r) y_r), conj(v_r) = u_r conj(scale) (1 for the leading row)
        sp += r == j + 1 ? y.x
                         : fma(uC[r].x, fma(cscC.x, y.x, -cscC.y * y.y), -uC[r].y * fma(cscC.x, y.y, cscC.y * y.x));
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
      // this CTA owns row j+1: publish its coefficients (and E = 2 Re(tau y)) before arriving
      const double2 y = row_y(0);
      double2 A, B, Q;
      coefs(first, j + 1, y, &A, &B, &Q);
      double2* rc = p.rowcoef + (j & 1) * 4;
      rc[0] = A;
      rc[1] = B;
      rc[2] = Q;
      rc[3] = make_double2(2.0 * fma(tauC.x, y.x, -tauC.y * y.y), 0.0);
    }
    if (jmodG == g) {   // the owner of row j stores u_j; k_eh_vscale forms v_j = conj(u_j) scale_j
      for (int c = j + 2 + tid; c < n; c += kTriThreads) p.vref[(size_t)j * n + c] = uC[c];
    }
    grid_arrive(p.bar);
    // local work while the other CTAs arrive: the own rows' coefficients for column j+1
    if (wid == 1) {
      for (int i = lane; i < Ra; i += 32) {
        const int lr = first + i, r = g + lr * G;
        double2 A, B, Q;
        coefs(lr, r, row_y(i), &A, &B, &Q);
        cA[lr] = A;
        cB[lr] = B;
        cQ[lr] = Q;
      }
    }
    tauAbs2 = fma(tauC.x, tauC.x, tauC.y * tauC.y);
    scP = scC;
    if (!grid_wait(p.bar, (unsigned)(G * (j + 1)), p.err)) return;
  }
}

}  // namespace
}  // namespace hpsi
