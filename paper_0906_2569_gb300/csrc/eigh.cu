// Lowest eigenpairs of a dense Hermitian matrix on the GPU, in float64: the reduced problem
// sum_k (H_jk - eps S_jk) c_k = 0 of the Rayleigh-Ritz step of block Davidson (paper App. A.2.1),
// where the reduced basis is orthonormal so S_jk is the identity.
//
//   1. Householder reduction Q^H A Q = T, Q = H_0 H_1 ... H_{n-2}, H_j = I - tau_j v_j v_j^H acting
//      on indices j+1..n-1 with v_j[j+1] = 1; T is real symmetric tridiagonal (diagonal d,
//      off-diagonal e).  Column j: H_j^H x = beta e_1 for the part x of the column below the
//      diagonal (beta real); then with y = A22 v_j, s = v_j^H y and w = tau_j y - |tau_j|^2 s v_j / 2
//      the trailing block becomes H_j^H A22 H_j = A22 - w v_j^H - v_j w^H.
//   2. The lowest nwant eigenvalues of T by multisection on Sturm counts.
//   3. Their eigenvectors z_i by inverse iteration.  Eigenvalues closer than 1e-10 |T| form a
//      cluster whose vectors are orthogonalised against each other (modified Gram-Schmidt) at each
//      iteration; the whole set is then orthonormalised by one Newton-Schulz step of the polar
//      decomposition (Z <- Z (3 I - Z^T Z) / 2), which mixes two vectors only in proportion to their
//      loss of orthogonality, itself of the order of rounding / gap, so residuals stay at rounding
//      level.
//   4. Back-transformation x_i = Q z_i = H_0 (H_1 (... (H_{n-2} z_i))), in blocks of 64 reflectors
//      written in compact WY form H_a ... H_b = I - V T V^H.  T^-1 = diag(1 / tau) +
//      strictly-upper(V^H V); one launch forms every block's T from it, and each block is then three
//      ZGEMMs (V^H X, T (V^H X), X - V (T V^H X)).
//
// Step 1 (eigh_tridiag.cuh) is one cooperative launch over G CTAs.  Row r of A lives in the shared memory of CTA
// r mod G for the whole reduction.  For column j every CTA rebuilds the same reflector from row j
// (A is Hermitian, so the column below the diagonal is the conjugate of the row's tail; the owner
// of row j published that row, updated, at the end of column j-1), updates its own rows with the
// previous column's w and v, and forms its rows of y = A22 v_j and its part of s.  One grid-wide
// barrier per column then publishes y, s and row j+1.  Every barrier wait is bounded in time: a
// wait that runs out raises the context's device error word and the kernel returns.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <string>

#include "hpsi_internal.h"
#include "eigh_tridiag.cuh"
#include "eigh_tridiag_real.cuh"
#include "eigh_tridiag_df.cuh"

namespace hpsi {

namespace {



// Gershgorin interval [lo, hi] of T, |T| bound and largest e^2, reduced over a warp.
__device__ void gershgorin(int n, const double* __restrict__ d, const double* __restrict__ e, double* lo, double* hi,
                           double* emax2) {
  const int lane = threadIdx.x & 31;
  double l = DBL_MAX, h = -DBL_MAX, m = 0.0;
  for (int k = lane; k < n; k += 32) {
    const double el = k > 0 ? fabs(e[k - 1]) : 0.0, er = k < n - 1 ? fabs(e[k]) : 0.0;
    l = fmin(l, d[k] - el - er);
    h = fmax(h, d[k] + el + er);
    m = fmax(m, er * er);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    l = fmin(l, __shfl_xor_sync(0xffffffffu, l, o));
    h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  }
  *lo = l;
  *hi = h;
  *emax2 = m;
}

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// Number of eigenvalues of T below sigma: the sign changes of the leading principal minors
// p_k of T - sigma I (p_k = (d_k - sigma) p_{k-1} - e_{k-1}^2 p_{k-2}).  Only the recurrence is
// float64; signs, zero tests and scaling work on the bit patterns (integer pipe).  A minor that is
// exactly zero becomes a tiny value of the sign opposite to the previous one (a pivmin-style
// perturbation of the diagonal); every 8 steps the pair is scaled by 2^-+400 through its exponent
// fields (a partner too small to scale down is negligible and flushed to zero; a subnormal is left
// as it is).
__device__ int sturm_count(int n, const double* __restrict__ d, const double* __restrict__ e2, double sigma) {
  constexpr long long kSign = (long long)0x8000000000000000ULL;
  constexpr long long kTiny = 0x0910000000000000LL;             // 2^-878
  constexpr long long kShift = 400LL << 52;
  double pm = 1.0, p = d[0] - sigma;
  if ((dbits(p) << 1) == 0) p = __longlong_as_double(kSign | kTiny);
  int cnt = dbits(p) < 0;
  auto step = [&](int k) {
    double pn = fma(d[k] - sigma, p, -e2[k - 1] * pm);
    if ((dbits(pn) << 1) == 0) pn = __longlong_as_double(((dbits(p) & kSign) ^ kSign) | kTiny);
    cnt += (dbits(pn) ^ dbits(p)) < 0;
    pm = p;
    p = pn;
  };
  int k = 1;
  for (; k + 8 <= n; k += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) step(k + u);
    const int ep = biased_exp(p), em = biased_exp(pm), ex = max(ep, em);
    if (ex > 1023 + 400) {
      p = __longlong_as_double(ep > 400 ? dbits(p) - kShift : dbits(p) & kSign);
      pm = __longlong_as_double(em > 400 ? dbits(pm) - kShift : dbits(pm) & kSign);
    } else if (ex < 1023 - 400) {
      if (ep > 0) p = __longlong_as_double(dbits(p) + kShift);
      if (em > 0) pm = __longlong_as_double(dbits(pm) + kShift);
    }
  }
  for (; k < n; ++k) step(k);
  return cnt;
}


// One CTA of kBisWarps warps per wanted eigenvalue i: (32 kBisWarps + 1)-way multisection of an
// interval with count(lo) <= i < count(hi), one Sturm count per thread and round, so the float64
// recurrences run on every sub-partition of the SM at once.
constexpr int kBisWarps = 1;   // 32 points per round: float64 Sturm counts are the bottleneck on this GPU, and
                                // 32 points take ~40% fewer of them than 64 for the same bracket width
__global__ void __launch_bounds__(32 * kBisWarps) k_eh_bisect(int n, const double* __restrict__ d,
                                                              const double* __restrict__ e,
                                                              const double* __restrict__ e2, int nwant,
                                                              double* __restrict__ lam) {
  constexpr int NP = 32 * kBisWarps;   // points per round
  __shared__ unsigned bal[kBisWarps];
  const int i = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (i >= nwant) return;
  double lo, hi, emax2;
  gershgorin(n, d, e, &lo, &hi, &emax2);
  const double tnorm = fmax(fmax(fabs(lo), fabs(hi)), DBL_MIN);
  const double pivmin = 1e-30 * fmax(1.0, emax2);
  lo -= 4.0 * DBL_EPSILON * tnorm + 4.0 * pivmin;
  hi += 4.0 * DBL_EPSILON * tnorm + 4.0 * pivmin;
  const double tol = 4.0 * DBL_EPSILON * tnorm;
  for (int round = 0; round < 64 && hi - lo > tol; ++round) {
    const double w = (hi - lo) / (double)(NP + 1);
    const int cnt = sturm_count(n, d, e2, lo + w * (double)(tid + 1));
    const unsigned above = __ballot_sync(0xffffffffu, cnt > i);
    if (lane == 0) bal[wid] = above;
    __syncthreads();
    int f = NP;   // index (point - 1) of the first point whose count exceeds i; NP if none
    for (int q = 0; q < kBisWarps; ++q)
      if (bal[q]) {
        f = 32 * q + __ffs(bal[q]) - 1;
        break;
      }
    __syncthreads();
    double nlo, nhi;
    if (f == NP) {
      nlo = lo + w * (double)NP;
      nhi = hi;
    } else {
      nlo = f > 0 ? lo + w * (double)f : lo;
      nhi = lo + w * (double)(f + 1);
    }
    if (nlo == lo && nhi == hi) break;   // the interval is down to a few ulps
    lo = nlo;
    hi = nhi;
  }
  if (tid == 0) lam[i] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double hash_unit(unsigned int i, unsigned int k) {
  unsigned int x = i * 0x9E3779B9u ^ (k * 0x85EBCA6Bu + 0x27D4EB2Fu);
  x ^= x >> 16;
  x *= 0x7FEB352Du;
  x ^= x >> 15;
  x *= 0x846CA68Bu;
  x ^= x >> 16;
  return (double)(x >> 8) * (1.0 / 16777216.0) - 0.5;
}

// z <- z - (zq . z) zq for the earlier members q of the cluster, then z /= |z|; whole warp.
__device__ bool orth_normalize(int n, double* z, const double* __restrict__ Z, int i0, int i) {
  const int lane = threadIdx.x & 31;
  for (int pass = 0; pass < 2; ++pass) {
    for (int q = i0; q < i; ++q) {
      const double* zq = Z + (size_t)q * n;
      double dot = 0.0;
      for (int k = lane; k < n; k += 32) dot += zq[k] * z[k];
      dot = warp_sum(dot);
      for (int k = lane; k < n; k += 32) z[k] -= dot * zq[k];
      __syncwarp();
    }
  }
  double nn = 0.0;
  for (int k = lane; k < n; k += 32) nn += z[k] * z[k];
  nn = warp_sum(nn);
  if (!(nn > 0.0) || !isfinite(nn)) return false;
  const double inv = 1.0 / sqrt(nn);
  for (int k = lane; k < n; k += 32) z[k] *= inv;
  __syncwarp();
  return true;
}

// One warp (one CTA) per cluster of the wanted eigenvalues; lane 0 factors T - lam I and runs the
// solves, the warp orthogonalises and normalises.  Vectors go to Z (column i, leading dim n).
// Inverse iteration for the eigenvalues without a neighbour within the cluster tolerance, one per
// lane: a float64 warp instruction costs the same with one active lane as with 32, so 32 of the
// serial tridiagonal recurrences share each instruction.  Per lane: T - lambda I = P L U with partial
// pivoting (the pivot choice as selects, the row interchanges as one ballot mask per step), then
// `iters` solves from a hashed start, normalised after each.  The factors and z live in a global
// scratch laid out [k][lane] per warp (5 n 32 doubles and n masks), so every step's accesses are
// coalesced.  Members of clusters are left to k_eh_invit.
__global__ void __launch_bounds__(32) k_eh_invit_lanes(int n, const double* __restrict__ d,
                                                       const double* __restrict__ e, int nwant,
                                                       const double* __restrict__ lam, double* __restrict__ Z,
                                                       double* __restrict__ scratch, int* __restrict__ status,
                                                       int iters) {
  const int lane = threadIdx.x, i = blockIdx.x * 32 + lane;
  double glo, ghi, emax2;
  gershgorin(n, d, e, &glo, &ghi, &emax2);
  double tnorm = fmax(fabs(glo), fabs(ghi));
  if (!(tnorm > 0.0)) tnorm = 1.0;
  const double ctol = 1e-10 * tnorm, tiny = DBL_EPSILON * tnorm;
  bool mine = i < nwant;
  if (mine && i > 0 && lam[i] - lam[i - 1] <= ctol) mine = false;
  if (mine && i + 1 < nwant && lam[i + 1] - lam[i] <= ctol) mine = false;
  if (__ballot_sync(0xffffffffu, mine) == 0u) return;
  const double li = mine ? lam[i] : lam[0];
  double* base = scratch + (size_t)blockIdx.x * ((size_t)5 * 32 * n + (n + 1) / 2);
  double* SL = base + lane;
  double* SU1 = SL + (size_t)32 * n;
  double* SU2 = SU1 + (size_t)32 * n;
  double* SU3 = SU2 + (size_t)32 * n;
  double* Zs = SU3 + (size_t)32 * n;
  unsigned* PIV = reinterpret_cast<unsigned*>(base + (size_t)5 * 32 * n);
  constexpr long long kMag = 0x7fffffffffffffffLL;
  auto guard = [&](double u) {
    return (__double_as_longlong(u) & kMag) < (__double_as_longlong(tiny) & kMag) ? (u < 0.0 ? -tiny : tiny) : u;
  };
  // every loop takes its independent loads kB steps at a time ahead of the dependent recurrence,
  // so that the L2 latency of the scratch is paid once per block, not once per step
  constexpr int kB = 8;
  double al = d[0] - li, be = n > 1 ? e[0] : 0.0;
  auto lu_step = [&](int k, double sub, double dk1, double cn) {
    const double dn = dk1 - li;
    const bool np = (__double_as_longlong(al) & kMag) >= (__double_as_longlong(sub) & kMag);
    const double ui = recip_nr(np ? guard(al) : sub);
    const double l = (np ? sub : al) * ui;
    SL[(size_t)k * 32] = l;
    SU1[(size_t)k * 32] = ui;
    SU2[(size_t)k * 32] = np ? be : dn;
    SU3[(size_t)k * 32] = np ? 0.0 : cn;
    const unsigned pv = __ballot_sync(0xffffffffu, !np);
    if (lane == 0) PIV[k] = pv;
    const double nal = fma(-l, np ? be : dn, np ? dn : be);
    be = np ? cn : -l * cn;
    al = nal;
  };
  int k = 0;
  for (; k + kB <= n - 1; k += kB) {
    double ev[kB], dv[kB], cv[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      ev[u] = e[k + u];
      dv[u] = d[k + u + 1];
      cv[u] = k + u + 1 < n - 1 ? e[k + u + 1] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) lu_step(k + u, ev[u], dv[u], cv[u]);
  }
  for (; k < n - 1; ++k) lu_step(k, e[k], d[k + 1], k + 1 < n - 1 ? e[k + 1] : 0.0);
  SU1[(size_t)(n - 1) * 32] = recip_nr(guard(al));
  double nn = 0.0;
  for (int q = 0; q < n; ++q) {
    const double v = hash_unit((unsigned)i, (unsigned)q);
    Zs[(size_t)q * 32] = v;
    nn = fma(v, v, nn);
  }
  bool ok = true;
  double sc = 1.0 / sqrt(nn);
  __syncwarp();
  for (int it = 0; it < iters; ++it) {
    // forward: row interchanges and L
    double zk = Zs[0] * sc;
    auto fwd_step = [&](int q, double z1r, double lq, unsigned pq) {
      const double z1 = z1r * sc;
      const bool sw = (pq >> lane) & 1u;
      const double a = sw ? z1 : zk, b = sw ? zk : z1;
      Zs[(size_t)q * 32] = a;
      zk = fma(-lq, a, b);
    };
    int q = 0;
    for (; q + kB <= n - 1; q += kB) {
      double zv[kB], lv[kB];
      unsigned pv[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        zv[u] = Zs[(size_t)(q + u + 1) * 32];
        lv[u] = SL[(size_t)(q + u) * 32];
        pv[u] = PIV[q + u];
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) fwd_step(q + u, zv[u], lv[u], pv[u]);
    }
    for (; q < n - 1; ++q) fwd_step(q, Zs[(size_t)(q + 1) * 32], SL[(size_t)q * 32], PIV[q]);
    // backward: U (three diagonals), with the squared norm of the result
    double z2 = zk * SU1[(size_t)(n - 1) * 32];
    Zs[(size_t)(n - 1) * 32] = z2;
    nn = z2 * z2;
    double z1 = 0.0;
    if (n >= 2) {
      z1 = (Zs[(size_t)(n - 2) * 32] - SU2[(size_t)(n - 2) * 32] * z2) * SU1[(size_t)(n - 2) * 32];
      Zs[(size_t)(n - 2) * 32] = z1;
      nn = fma(z1, z1, nn);
    }
    auto bwd_step = [&](int q, double zq, double u1, double u2, double u3) {
      const double zz = (zq - u2 * z1 - u3 * z2) * u1;
      Zs[(size_t)q * 32] = zz;
      nn = fma(zz, zz, nn);
      z2 = z1;
      z1 = zz;
    };
    q = n - 3;
    for (; q - kB + 1 >= 0; q -= kB) {
      double zv[kB], a1[kB], a2[kB], a3[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        const size_t o = (size_t)(q - u) * 32;
        zv[u] = Zs[o];
        a1[u] = SU1[o];
        a2[u] = SU2[o];
        a3[u] = SU3[o];
      }
#pragma unroll
      for (int u = 0; u < kB; ++u) bwd_step(q - u, zv[u], a1[u], a2[u], a3[u]);
    }
    for (; q >= 0; --q) {
      const size_t o = (size_t)q * 32;
      bwd_step(q, Zs[o], SU1[o], SU2[o], SU3[o]);
    }
    if (!(nn > 0.0) || !isfinite(nn)) ok = false;
    sc = ok ? 1.0 / sqrt(nn) : 1.0;
  }
  if (!mine) return;
  if (!ok) {
    atomicExch(status, 1);
    return;
  }
  double* zi = Z + (size_t)i * n;
  for (int k = 0; k < n; ++k) zi[k] = Zs[(size_t)k * 32] * sc;
}

__global__ void __launch_bounds__(32) k_eh_invit(int n, const double* __restrict__ d, const double* __restrict__ e,
                                                 int nwant, const double* __restrict__ lam, double* __restrict__ Z,
                                                 int* __restrict__ status, int skip_single, int iters) {
  extern __shared__ double sh[];
  double* sd = sh;
  double* se = sd + n;
  double* sl = se + n;
  double* su1 = sl + n;   // reciprocals of U's diagonal
  double* su2 = su1 + n;
  double* su3 = su2 + n;
  double* z = su3 + n;
  unsigned char* spv = reinterpret_cast<unsigned char*>(z + n);
  const int i0 = blockIdx.x, lane = threadIdx.x;
  if (i0 >= nwant) return;
  double glo, ghi, emax2;
  gershgorin(n, d, e, &glo, &ghi, &emax2);
  double tnorm = fmax(fabs(glo), fabs(ghi));
  if (!(tnorm > 0.0)) tnorm = 1.0;
  const double ctol = 1e-10 * tnorm;
  if (i0 > 0 && lam[i0] - lam[i0 - 1] <= ctol) return;   // not the first of its cluster
  if (skip_single && (i0 + 1 >= nwant || lam[i0 + 1] - lam[i0] > ctol)) return;   // k_eh_invit_lanes has it
  for (int k = lane; k < n; k += 32) {
    sd[k] = d[k];
    se[k] = k < n - 1 ? e[k] : 0.0;
  }
  __syncwarp();
  const double tiny = DBL_EPSILON * tnorm;
  for (int i = i0; i < nwant && (i == i0 || lam[i] - lam[i - 1] <= ctol); ++i) {
    const double li = lam[i];
    if (lane == 0) {
      // T - li I = P L U by Gaussian elimination with row interchanges (|.| compared on bits)
      constexpr long long kMag = 0x7fffffffffffffffLL;
      double al = sd[0] - li, be = n > 1 ? se[0] : 0.0;
      for (int k = 0; k < n - 1; ++k) {
        const double sub = se[k], dn = sd[k + 1] - li, cn = k + 1 < n - 1 ? se[k + 1] : 0.0;
        if ((__double_as_longlong(al) & kMag) >= (__double_as_longlong(sub) & kMag)) {
          double u = al;
          if ((__double_as_longlong(u) & kMag) < (__double_as_longlong(tiny) & kMag)) u = u < 0.0 ? -tiny : tiny;
          const double ui = recip_nr(u);
          const double l = sub * ui;
          sl[k] = l;
          spv[k] = 0;
          su1[k] = ui;
          su2[k] = be;
          su3[k] = 0.0;
          al = fma(-l, be, dn);
          be = cn;
        } else {
          const double ui = recip_nr(sub);
          const double l = al * ui;
          sl[k] = l;
          spv[k] = 1;
          su1[k] = ui;
          su2[k] = dn;
          su3[k] = cn;
          al = fma(-l, dn, be);
          be = -l * cn;
        }
      }
      double u = al;
      if ((__double_as_longlong(u) & kMag) < (__double_as_longlong(tiny) & kMag)) u = u < 0.0 ? -tiny : tiny;
      su1[n - 1] = recip_nr(u);
    }
    for (int k = lane; k < n; k += 32) z[k] = hash_unit((unsigned)i, (unsigned)k);
    __syncwarp();
    bool ok = orth_normalize(n, z, Z, i0, i);
    for (int it = 0; it < iters && ok; ++it) {
      if (lane == 0) {
        for (int k = 0; k < n - 1; ++k) {
          if (spv[k]) {
            const double t = z[k];
            z[k] = z[k + 1];
            z[k + 1] = t;
          }
          z[k + 1] -= sl[k] * z[k];
        }
        z[n - 1] *= su1[n - 1];
        if (n >= 2) z[n - 2] = (z[n - 2] - su2[n - 2] * z[n - 1]) * su1[n - 2];
        for (int k = n - 3; k >= 0; --k) z[k] = (z[k] - su2[k] * z[k + 1] - su3[k] * z[k + 2]) * su1[k];
      }
      __syncwarp();
      ok = orth_normalize(n, z, Z, i0, i);
    }
    if (!ok) {
      if (lane == 0) atomicExch(status, 1);
      return;
    }
    double* zi = Z + (size_t)i * n;
    for (int k = lane; k < n; k += 32) zi[k] = z[k];
    __syncwarp();
  }
}

constexpr int kWY = 64;   // reflectors per compact-WY block of the back-transformation
constexpr int kMaxCtas = 1024;   // CTAs of a reduction at most (one per SM)
constexpr int kWYRows = kWY / 32;   // rows of a block per lane in the back substitution

// v_j[c] = conj(u_j[c]) scale_j for c > j + 1 and v_j[j + 1] = 1, in place (rows j < n - 1).
__global__ void k_eh_vscale(int n, const double2* __restrict__ vscale, double2* __restrict__ vref) {
  const int j = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n - 1 || c <= j || c >= n) return;
  double2* v = vref + (size_t)j * n + c;
  if (c == j + 1) {
    *v = make_double2(1.0, 0.0);
    return;
  }
  const double2 u = *v, sc = vscale[j];
  *v = make_double2(fma(sc.x, u.x, sc.y * u.y), fma(sc.y, u.x, -sc.x * u.y));
}

// status[0] = 1 when some |G_ij - delta_ij| exceeds tol (G = Z^T Z, nwant x nwant)
template <typename T>
__global__ void k_eh_orthcheck(int nw, const T* __restrict__ G, double tol, int* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nw * nw) return;
  const double g = (double)G[i] - ((i % nw) == (i / nw) ? 1.0 : 0.0);
  if (!(fabs(g) <= tol)) atomicExch(status, 1);
}

// out = in, element type converted (grid-stride)
template <typename A, typename B>
__global__ void k_eh_cvt(size_t n, const A* __restrict__ in, B* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (B)in[i];
}

inline int cvt_grid(size_t n) { return (int)std::min<size_t>(4096, (n + 255) / 256); }

// x = z (real eigenvectors of T into the complex output, column-major, leading dim n)
__global__ void k_eh_widen(int n, int nwant, const double* __restrict__ Z, double2* __restrict__ X) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n * nwant) return;
  X[idx] = make_double2(Z[idx], 0.0);
}

// The upper-triangular factor of a compact-WY block, H_{k nb} ... H_{k nb + nb - 1} = I - V T V^H,
// has the inverse S = T^-1 = diag(1 / tau_i) + (strictly upper part of G = V^H V), so
// T = (I + diag(tau) striu(G))^-1 diag(tau): a back substitution y_q = tau_q (w_q - sum_{r > q} S_qr y_r)
// applied to the columns w = e_c of the identity.  It needs no division and gives a zero row and
// column for an identity reflector (tau_q = 0).  Grid (kWY / 4, blocks): one warp per column of one
// block's T; lane l holds rows l, l + 32, ...; rows are finalised from the last one, each
// subtracting its contribution from the rows above.  G holds the blocks' Gram matrices and T receives
// the factors (both column-major kWY x kWY per block; only the strictly upper part of G is read).
__global__ void __launch_bounds__(128) k_eh_tfactor(const double2* __restrict__ Gall, const double2* __restrict__ tauall,
                                                    double2* __restrict__ Tall) {
  extern __shared__ double2 gs[];   // strictly upper part of G, column q at q (q - 1) / 2
  const size_t blk = (size_t)blockIdx.y * kWY * kWY;
  const double2* G = Gall + blk;
  const double2* tau = tauall + (size_t)blockIdx.y * kWY;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < kWY * (kWY - 1) / 2; idx += blockDim.x) {
    int q = (int)(0.5f * (1.0f + sqrtf(1.0f + 8.0f * (float)idx)));   // column: q (q - 1) / 2 <= idx
    while (q * (q - 1) / 2 > idx) --q;
    while ((q + 1) * q / 2 <= idx) ++q;
    gs[idx] = G[(idx - q * (q - 1) / 2) + (size_t)q * kWY];
  }
  __syncthreads();
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= kWY) return;
  double2 acc[kWYRows];   // right-hand side rows lane + 32 s, reduced as rows finalise
#pragma unroll
  for (int sl = 0; sl < kWYRows; ++sl) acc[sl] = make_double2(lane + 32 * sl == col ? 1.0 : 0.0, 0.0);
  for (int q = kWY - 1; q >= 0; --q) {
    // the owner finalises y_q = tau_q acc_q, then every row r < q subtracts S_rq y_q
    const int own = q & 31, oslot = q >> 5;
    double2 yq = make_double2(0.0, 0.0);
    if (lane == own) {
      const double2 t = tau[q];
#pragma unroll
      for (int sl = 0; sl < kWYRows; ++sl)
        if (sl == oslot) {
          const double2 a = acc[sl];
          yq = make_double2(t.x * a.x - t.y * a.y, t.x * a.y + t.y * a.x);
          acc[sl] = yq;
        }
    }
    yq.x = __shfl_sync(0xffffffffu, yq.x, own);
    yq.y = __shfl_sync(0xffffffffu, yq.y, own);
    const double2* gq = gs + q * (q - 1) / 2;
#pragma unroll
    for (int sl = 0; sl < kWYRows; ++sl) {
      if (32 * sl < q) {   // warp-uniform: some row of this slot lies above q
        const int r = lane + 32 * sl;
        if (r < q) {
          const double2 g = gq[r];
          acc[sl].x -= g.x * yq.x - g.y * yq.y;
          acc[sl].y -= g.x * yq.y + g.y * yq.x;
        }
      }
    }
  }
  double2* t = Tall + blk + (size_t)col * kWY;
#pragma unroll
  for (int sl = 0; sl < kWYRows; ++sl) t[lane + 32 * sl] = acc[sl];
}

constexpr size_t kTrsvSmem = sizeof(double2) * (size_t)kWY * (kWY - 1) / 2;

// Real forms of the two back-transformation helpers (the reduction of a real symmetric matrix):
// v_j[c] = u_j[c] scale_j for c > j + 1 and v_j[j + 1] = 1.
__global__ void k_eh_vscale_r(int n, const double* __restrict__ vscale, double* __restrict__ vref) {
  const int j = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n - 1 || c <= j || c >= n) return;
  double* v = vref + (size_t)j * n + c;
  *v = c == j + 1 ? 1.0 : *v * vscale[j];
}

// After a double-float reduction: tau_j = 2 / (v_j^T v_j) from the diagonal of the blocks' Gram
// matrices (the reduction's tau agrees to ~1e-14), so that every reflector I - tau v v^T is
// orthogonal to float64 rounding; a zero tau (no reflection) stays zero.
__global__ void k_eh_tau_fix(int nref, const double* __restrict__ Gall, double* __restrict__ tau) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nref || tau[j] == 0.0) return;
  const int k = j / kWY, jj = j % kWY;
  tau[j] = 2.0 / Gall[(size_t)k * kWY * kWY + (size_t)jj * kWY + jj];
}

// T of a real compact-WY block from G = V^T V and tau, as k_eh_tfactor does for complex blocks.
__global__ void __launch_bounds__(128) k_eh_tfactor_r(const double* __restrict__ Gall, const double* __restrict__ tauall,
                                                      double* __restrict__ Tall) {
  extern __shared__ double gsr[];   // strictly upper part of G, column q at q (q - 1) / 2
  const size_t blk = (size_t)blockIdx.y * kWY * kWY;
  const double* G = Gall + blk;
  const double* tau = tauall + (size_t)blockIdx.y * kWY;
  for (int idx = threadIdx.x; idx < kWY * (kWY - 1) / 2; idx += blockDim.x) {
    int q = (int)(0.5f * (1.0f + sqrtf(1.0f + 8.0f * (float)idx)));
    while (q * (q - 1) / 2 > idx) --q;
    while ((q + 1) * q / 2 <= idx) ++q;
    gsr[idx] = G[(idx - q * (q - 1) / 2) + (size_t)q * kWY];
  }
  __syncthreads();
  const int col = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (col >= kWY) return;
  double acc[kWYRows];
#pragma unroll
  for (int sl = 0; sl < kWYRows; ++sl) acc[sl] = lane + 32 * sl == col ? 1.0 : 0.0;
  for (int q = kWY - 1; q >= 0; --q) {
    const int own = q & 31, oslot = q >> 5;
    double yq = 0.0;
    if (lane == own) {
#pragma unroll
      for (int sl = 0; sl < kWYRows; ++sl)
        if (sl == oslot) {
          yq = tau[q] * acc[sl];
          acc[sl] = yq;
        }
    }
    yq = __shfl_sync(0xffffffffu, yq, own);
    const double* gq = gsr + q * (q - 1) / 2;
#pragma unroll
    for (int sl = 0; sl < kWYRows; ++sl) {
      if (32 * sl < q) {
        const int r = lane + 32 * sl;
        if (r < q) acc[sl] = fma(-gq[r], yq, acc[sl]);
      }
    }
  }
  double* t = Tall + blk + (size_t)col * kWY;
#pragma unroll
  for (int sl = 0; sl < kWYRows; ++sl) t[lane + 32 * sl] = acc[sl];
}

struct EighState {
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t solver = nullptr;
  int ncap = 0, wcap = 0;
  double *d = nullptr, *e = nullptr, *e2 = nullptr, *sacc = nullptr, *lam = nullptr, *Z = nullptr, *Z2 = nullptr;
  double* spart = nullptr;   // [2][kMaxCtas] the double-float reduction's per-CTA parts of s
  double* invs = nullptr;    // k_eh_invit_lanes scratch
  size_t invcap = 0;
  double* gram = nullptr;
  double2 *tau = nullptr, *vref = nullptr, *ybuf = nullptr, *rnext = nullptr, *rowcoef = nullptr, *vscale = nullptr;
  double2 *wgram = nullptr, *tfac = nullptr, *w1 = nullptr, *w2 = nullptr;   // compact-WY blocks
  unsigned int* bar = nullptr;
  int* info = nullptr;    // [0] orthogonality check of the eigenvectors, [1] inverse-iteration status
  // cuSOLVER zheevdx path
  int zcap = 0, zlwork = 0;
  double2 *acopy = nullptr, *zwork = nullptr;
  double* wfull = nullptr;
  int* zinfo = nullptr;
};

void free_state(EighState& s) {
  void* ptrs[] = {s.d,    s.e,     s.e2,    s.sacc,    s.lam,   s.Z,  s.gram, s.tau,
                  s.vref, s.ybuf,  s.rnext, s.rowcoef, s.wgram, s.w1, s.bar,  s.info, s.vscale, s.Z2, s.tfac, s.w2,
                  s.spart};
  for (void* q : ptrs) cudaFree(q);
  cudaFree(s.invs);
  const EighState keep = s;
  s = EighState{};
  s.blas = keep.blas;
  s.solver = keep.solver;
  s.zcap = keep.zcap;
  s.zlwork = keep.zlwork;
  s.acopy = keep.acopy;
  s.zwork = keep.zwork;
  s.wfull = keep.wfull;
  s.zinfo = keep.zinfo;
}

void free_zheevdx(EighState& s) {
  cudaFree(s.acopy);
  cudaFree(s.zwork);
  cudaFree(s.wfull);
  cudaFree(s.zinfo);
  s.acopy = s.zwork = nullptr;
  s.wfull = nullptr;
  s.zinfo = nullptr;
  s.zcap = s.zlwork = 0;
}

int grow(Context& c, EighState& s, int n, int nwant) {
  if (n <= s.ncap && nwant <= s.wcap) return HPSI_OK;
  const int ncap0 = s.ncap, wcap0 = s.wcap;
  free_state(s);
  s.ncap = ncap0;
  s.wcap = wcap0;
  const int N = std::max(n, s.ncap), W = std::max(nwant, s.wcap);
  bool ok = true;
  auto al = [&](void** q, size_t bytes) { ok = ok && cudaMalloc(q, std::max<size_t>(bytes, 16)) == cudaSuccess; };
  al((void**)&s.d, sizeof(double) * N);
  al((void**)&s.e, sizeof(double) * N);
  al((void**)&s.e2, sizeof(double) * N);
  al((void**)&s.sacc, sizeof(double) * 4);
  al((void**)&s.rowcoef, sizeof(double2) * 8);
  al((void**)&s.spart, sizeof(double) * 2 * kMaxCtas);
  al((void**)&s.vscale, sizeof(double2) * N);
  al((void**)&s.lam, sizeof(double) * W);
  al((void**)&s.Z, sizeof(double) * (size_t)N * W);
  al((void**)&s.Z2, sizeof(double) * (size_t)N * W);
  al((void**)&s.gram, sizeof(double) * (size_t)W * W);
  const int K = (N + kWY - 1) / kWY;
  al((void**)&s.tau, sizeof(double2) * (N + kWY));
  al((void**)&s.vref, sizeof(double2) * (size_t)(N + kWY) * N);
  al((void**)&s.wgram, sizeof(double2) * (size_t)K * kWY * kWY);
  al((void**)&s.tfac, sizeof(double2) * (size_t)K * kWY * kWY);
  al((void**)&s.w1, sizeof(double2) * (size_t)kWY * W);
  al((void**)&s.w2, sizeof(double2) * (size_t)kWY * W);
  al((void**)&s.ybuf, sizeof(double2) * 2 * N);
  al((void**)&s.rnext, sizeof(double2) * 2 * N);
  al((void**)&s.bar, sizeof(unsigned int) * 64);
  al((void**)&s.info, sizeof(int) * 2);
  if (!ok) {
    free_state(s);
    return fail(c, HPSI_ENOMEM, "eigensolver workspace allocation failed");
  }
  s.ncap = N;
  s.wcap = W;
  return HPSI_OK;
}

// Eigenvectors of T for the lowest nwant eigenvalues in s.lam: one lane per isolated eigenvalue
// (k_eh_invit_lanes), one warp per cluster of close ones (k_eh_invit).  Vectors to s.Z.  iters
// solves from a random start: a neighbour at a gap g just above the cluster tolerance keeps a share
// (4 eps |T| / g)^iters, ~1e-5 after two solves, which one Newton-Schulz step only squares; three
// solves for float64 eigenvectors, two for float32 ones.
int invit_all(Context& c, EighState& s, int n, int nwant, int iters) {
  const int nblk = (nwant + 31) / 32;
  const size_t per = (size_t)5 * 32 * n + (n + 1) / 2;
  const size_t need = sizeof(double) * per * nblk;
  if (need > s.invcap) {
    cudaFree(s.invs);
    s.invs = nullptr;
    s.invcap = 0;
    if (cudaMalloc((void**)&s.invs, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, HPSI_ENOMEM, "inverse-iteration scratch allocation failed");
    }
    s.invcap = need;
  }
  HPSI_LAUNCH(c, HPSI_K_EIGH, (k_eh_invit_lanes<<<nblk, 32, 0, c.stream>>>(n, s.d, s.e, nwant, s.lam, s.Z, s.invs,
                                                                          s.info + 1, iters)));
  const size_t ismem = sizeof(double) * 7 * (size_t)n + (size_t)n + 16;
  if (ismem > 48 * 1024) {
    const cudaError_t err = cudaFuncSetAttribute(k_eh_invit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ismem);
    if (err != cudaSuccess) return cuda_fail(c, err, "inverse iteration: smem attribute");
  }
  HPSI_LAUNCH(c, HPSI_K_EIGH,
              (k_eh_invit<<<nwant, 32, ismem, c.stream>>>(n, s.d, s.e, nwant, s.lam, s.Z, s.info + 1, 1, iters)));
  return HPSI_OK;
}

int ensure_state(Context& c, EighState** out) {
  EighState* s = reinterpret_cast<EighState*>(c.eigh);
  if (!s) {
    s = new EighState();
    c.eigh = s;
    if (cublasCreate(&s->blas) != CUBLAS_STATUS_SUCCESS) return fail(c, HPSI_ECUDA, "eigensolver: cublasCreate failed");
    if (cusolverDnCreate(&s->solver) != CUSOLVER_STATUS_SUCCESS)
      return fail(c, HPSI_ECUDA, "eigensolver: cusolverDnCreate failed");
  }
  cublasSetStream(s->blas, c.stream);
  cusolverDnSetStream(s->solver, c.stream);
  *out = s;
  return HPSI_OK;
}

// cuSOLVER zheevdx on a copy of the matrix: lowest nwant pairs.
int eigh_zheevdx(Context& c, EighState& s, const double2* a, int lda, int n, int nwant, double* w_out,
                 double2* v_out) {
  if (n > s.zcap) {
    free_zheevdx(s);
    int lw = 0, meig = 0;
    if (cudaMalloc((void**)&s.acopy, sizeof(double2) * (size_t)n * n) != cudaSuccess ||
        cudaMalloc((void**)&s.wfull, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc((void**)&s.zinfo, sizeof(int)) != cudaSuccess) {
      free_zheevdx(s);
      return fail(c, HPSI_ENOMEM, "eigensolver: zheevdx workspace allocation failed");
    }
    if (cusolverDnZheevdx_bufferSize(s.solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I,
                                     CUBLAS_FILL_MODE_UPPER, n, reinterpret_cast<cuDoubleComplex*>(s.acopy), n, 0.0,
                                     0.0, 1, n, &meig, s.wfull, &lw) != CUSOLVER_STATUS_SUCCESS) {
      free_zheevdx(s);
      return fail(c, HPSI_ECUDA, "eigensolver: zheevdx buffer size failed");
    }
    s.zlwork = std::max(lw, 1);
    if (cudaMalloc((void**)&s.zwork, sizeof(double2) * s.zlwork) != cudaSuccess) {
      free_zheevdx(s);
      return fail(c, HPSI_ENOMEM, "eigensolver: zheevdx workspace allocation failed");
    }
    s.zcap = n;
  }
  cudaError_t err = cudaMemcpy2DAsync(s.acopy, sizeof(double2) * n, a, sizeof(double2) * lda, sizeof(double2) * n, n,
                                      cudaMemcpyDeviceToDevice, c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigensolver: matrix copy");
  int meig = 0;
  if (cusolverDnZheevdx(s.solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_UPPER, n,
                        reinterpret_cast<cuDoubleComplex*>(s.acopy), n, 0.0, 0.0, 1, nwant, &meig, s.wfull,
                        reinterpret_cast<cuDoubleComplex*>(s.zwork), s.zlwork, s.zinfo) != CUSOLVER_STATUS_SUCCESS)
    return fail(c, HPSI_ECUDA, "eigensolver: cusolverDnZheevdx failed");
  err = cudaMemcpyAsync(w_out, s.wfull, sizeof(double) * nwant, cudaMemcpyDeviceToDevice, c.stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(v_out, s.acopy, sizeof(double2) * (size_t)n * nwant, cudaMemcpyDeviceToDevice, c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigensolver: result copy");
  int info = 0;
  err = cudaMemcpyAsync(&info, s.zinfo, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigensolver: zheevdx");
  if (info != 0 || meig < nwant)
    return fail(c, HPSI_ESINGULAR, "zheevdx of the reduced matrix failed, info " + std::to_string(info));
  return HPSI_OK;
}

int tri_ctas(const Context& c, int n) {
  int G = std::min(std::min(c.sm_count, kMaxCtas), std::max(8, (n + 3) / 4));
  return std::max(1, std::min(G, n));
}

size_t tri_smem(int n, int G) {
  const int R = (n + G - 1) / G;
  return sizeof(double2) * ((size_t)(3 + R) * n + 8 * (size_t)R);
}

size_t tri_smem_r(int n, int G) {
  const int R = (n + G - 1) / G;
  return sizeof(double) * ((size_t)(3 + R) * n + 8 * (size_t)R);
}

}  // namespace

bool eigh_supported(const Context& c, int n) {
  if (n < 1 || n > kMaxN) return false;
  return tri_smem(n, tri_ctas(c, n)) <= c.smem_optin;
}

void eigh_release(Context& c) {
  EighState* s = reinterpret_cast<EighState*>(c.eigh);
  if (!s) return;
  free_state(*s);
  free_zheevdx(*s);
  if (s->blas) cublasDestroy(s->blas);
  if (s->solver) cusolverDnDestroy(s->solver);
  delete s;
  c.eigh = nullptr;
}

int eigh_lowest(Context& c, const double2* a, int lda, int n, int nwant, double* w_out, double2* v_out,
                bool* fallback) {
  *fallback = false;
  if (n < 1 || nwant < 1 || nwant > n || lda < n) return fail(c, HPSI_EINVAL, "eigh_lowest: bad sizes");
  if (!eigh_supported(c, n)) {
    *fallback = true;
    return HPSI_OK;
  }
  EighState* s = nullptr;
  int rc = ensure_state(c, &s);
  if (rc) return rc;
  rc = grow(c, *s, n, nwant);
  if (rc) return rc;
  cudaError_t err;

  // 1. tridiagonal reduction (cooperative)
  const int G = tri_ctas(c, n);
  const size_t smem = tri_smem(n, G);
  err = cudaFuncSetAttribute(k_eh_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest: smem attribute");
  err = cudaMemsetAsync(s->bar, 0, sizeof(unsigned int) * 64, c.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(s->vref, 0, sizeof(double2) * (size_t)(n + kWY) * n, c.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(s->tau, 0, sizeof(double2) * (n + kWY), c.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(s->sacc, 0, sizeof(double) * 4, c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest: workspace reset");
  err = cudaMemsetAsync(s->info, 0, sizeof(int) * 2, c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest: status reset");
  TriArgs ta{n, lda, G, a, s->d, s->e, s->e2, s->tau, s->vref, s->ybuf, s->rnext, s->rowcoef, s->vscale, s->sacc, s->bar,
             c.d_err};
  void* args[] = {&ta};
  HPSI_LAUNCH(c, HPSI_K_TRIDIAG,
              (err = cudaLaunchCooperativeKernel((const void*)k_eh_tridiag, dim3(G), dim3(kTriThreads), args, smem,
                                                 c.stream)));
  ++c.tri_calls;
  c.tri_flops += 16.0 / 3.0 * (double)n * (double)n * (double)n;
  if (err == cudaErrorCooperativeLaunchTooLarge) {   // the device cannot hold the grid at once
    cudaGetLastError();
    *fallback = true;
    return HPSI_OK;
  }
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest: tridiagonal reduction launch");
  // 2. eigenvalues
  HPSI_LAUNCH(c, HPSI_K_EIGH,
              (k_eh_bisect<<<nwant, 32 * kBisWarps, 0, c.stream>>>(n, s->d, s->e, s->e2, nwant, s->lam)));
  // 3. eigenvectors of T
  rc = invit_all(c, *s, n, nwant, 3);
  if (rc) return rc;
  //    orthonormalisation of Z by one Newton-Schulz step of the polar decomposition,
  //    Z <- Z (3 I - Z^T Z) / 2: inverse iteration leaves |Z^T Z - I| at rounding / gap (below
  //    1e-6 for gaps above the cluster tolerance), which one step squares; a larger departure
  //    (a lost vector) makes the caller fall back to cuSOLVER
  const double one = 1.0, zero = 0.0, mhalf = -0.5, three_half = 1.5;
  if (cublasDgemm(s->blas, CUBLAS_OP_T, CUBLAS_OP_N, nwant, nwant, n, &one, s->Z, n, s->Z, n, &zero, s->gram, nwant) !=
      CUBLAS_STATUS_SUCCESS)
    return fail(c, HPSI_ECUDA, "eigh_lowest: Gram matrix of the eigenvectors failed");
  HPSI_LAUNCH(c, HPSI_K_EIGH,
              (k_eh_orthcheck<double><<<(nwant * nwant + 255) / 256, 256, 0, c.stream>>>(nwant, s->gram, 1e-4, s->info)));
  if (cudaMemcpyAsync(s->Z2, s->Z, sizeof(double) * (size_t)n * nwant, cudaMemcpyDeviceToDevice, c.stream) !=
          cudaSuccess ||
      cublasDgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, nwant, nwant, &mhalf, s->Z, n, s->gram, nwant, &three_half,
                  s->Z2, n) != CUBLAS_STATUS_SUCCESS)
    return fail(c, HPSI_ECUDA, "eigh_lowest: Newton-Schulz step failed");
  if (n > 1) HPSI_LAUNCH(c, HPSI_K_EIGH, (k_eh_vscale<<<dim3((n + 255) / 256, n - 1), 256, 0, c.stream>>>(n, s->vscale, s->vref)));
  // 4. back-transformation, one compact-WY block of kWY reflectors at a time from the last:
  //    X <- (I - V_k T_k V_k^H) X over rows k kWY + 1 .. n-1 (reflectors past n-2 are zero)
  HPSI_LAUNCH(c, HPSI_K_EIGH,
              (k_eh_widen<<<(unsigned)(((size_t)n * nwant + 255) / 256), 256, 0, c.stream>>>(n, nwant, s->Z2, v_out)));
  if (n > 1) {
    const int K = (n - 1 + kWY - 1) / kWY;
    const cuDoubleComplex zone = make_cuDoubleComplex(1.0, 0.0), zzero = make_cuDoubleComplex(0.0, 0.0),
                          zmone = make_cuDoubleComplex(-1.0, 0.0);
    auto Zc = [](double2* q) { return reinterpret_cast<cuDoubleComplex*>(q); };
    if (cublasZgemmStridedBatched(s->blas, CUBLAS_OP_C, CUBLAS_OP_N, kWY, kWY, n - 1, &zone, Zc(s->vref + 1), n,
                                  (long long)kWY * n, Zc(s->vref + 1), n, (long long)kWY * n, &zzero, Zc(s->wgram),
                                  kWY, (long long)kWY * kWY, K) != CUBLAS_STATUS_SUCCESS)
      return fail(c, HPSI_ECUDA, "eigh_lowest: reflector Gram matrices failed");
    err = cudaFuncSetAttribute(k_eh_tfactor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrsvSmem);
    if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest: smem attribute");
    HPSI_LAUNCH(c, HPSI_K_EIGH,
                (k_eh_tfactor<<<dim3(kWY / 4, K), 128, kTrsvSmem, c.stream>>>(s->wgram, s->tau, s->tfac)));
    for (int k = K - 1; k >= 0; --k) {
      const int r0 = k * kWY + 1, m = n - r0;
      double2* V = s->vref + (size_t)k * kWY * n + r0;
      if (cublasZgemm(s->blas, CUBLAS_OP_C, CUBLAS_OP_N, kWY, nwant, m, &zone, Zc(V), n, Zc(v_out + r0), n, &zzero,
                      Zc(s->w1), kWY) != CUBLAS_STATUS_SUCCESS ||
          cublasZgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, kWY, nwant, kWY, &zone, Zc(s->tfac + (size_t)k * kWY * kWY),
                      kWY, Zc(s->w1), kWY, &zzero, Zc(s->w2), kWY) != CUBLAS_STATUS_SUCCESS ||
          cublasZgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, m, nwant, kWY, &zmone, Zc(V), n, Zc(s->w2), kWY, &zone,
                      Zc(v_out + r0), n) != CUBLAS_STATUS_SUCCESS)
        return fail(c, HPSI_ECUDA, "eigh_lowest: back-transformation GEMM failed");
    }
  }
  err = cudaMemcpyAsync(w_out, s->lam, sizeof(double) * nwant, cudaMemcpyDeviceToDevice, c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest: eigenvalue copy");
  int info[2] = {0, 0};
  err = cudaMemcpyAsync(info, s->info, sizeof(int) * 2, cudaMemcpyDeviceToHost, c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest: status copy");
  rc = check_device_error(c);
  if (rc) return rc;
  ++c.eig_calls;
  if (info[0] != 0 || info[1] != 0) {   // inverse iteration lost a vector: the caller falls back
    *fallback = true;
    ++c.eig_fallbacks;
  }
  return HPSI_OK;
}

bool eigh_supported_real(const Context& c, int n) {
  if (n < 1 || n > kMaxNR) return false;
  return tri_smem_r(n, tri_ctas(c, n)) <= c.smem_optin;
}

// The same four steps for a real symmetric matrix (float64, column-major, upper triangle read):
// real Householder reduction, multisection and inverse iteration on T, real compact-WY
// back-transformation by DGEMMs.  Eigenvectors go to v_out [nwant][n] (column-major, ld n).
// vec32: the eigenvectors are wanted to float32 accuracy only (a float32 basis is rotated by them),
// so their Gram matrix, the Newton-Schulz step and the back-transformation run as float32 GEMMs on
// float32 copies (FP32 throughput is ~64x FP64 on GB300); the eigenvalues and the inverse iteration
// stay float64.  df: the reduction's row work in double-float arithmetic (k_eh_tridiag_df, ~1e-13
// relative) instead of float64.
int eigh_lowest_real(Context& c, const double* a, int lda, int n, int nwant, double* w_out, double* v_out,
                     bool* fallback, bool vec32, bool df) {
  *fallback = false;
  if (n < 1 || nwant < 1 || nwant > n || lda < n) return fail(c, HPSI_EINVAL, "eigh_lowest_real: bad sizes");
  if (!eigh_supported_real(c, n)) {
    *fallback = true;
    return HPSI_OK;
  }
  EighState* s = nullptr;
  int rc = ensure_state(c, &s);
  if (rc) return rc;
  rc = grow(c, *s, n, nwant);
  if (rc) return rc;
  cudaError_t err;
  // the complex work buffers are reused as real ones (each holds at least twice the doubles needed)
  double* tau = reinterpret_cast<double*>(s->tau);
  double* vref = reinterpret_cast<double*>(s->vref);
  double* vscale = reinterpret_cast<double*>(s->vscale);
  double* wgram = reinterpret_cast<double*>(s->wgram);
  double* tfac = reinterpret_cast<double*>(s->tfac);
  double* w1 = reinterpret_cast<double*>(s->w1);
  double* w2 = reinterpret_cast<double*>(s->w2);

  // 1. tridiagonal reduction (cooperative)
  const int G = tri_ctas(c, n);
  const size_t smem = tri_smem_r(n, G);
  const void* tri_kernel = df ? (const void*)k_eh_tridiag_df : (const void*)k_eh_tridiag_r;
  err = cudaFuncSetAttribute(tri_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest_real: smem attribute");
  err = cudaMemsetAsync(s->bar, 0, sizeof(unsigned int) * 64, c.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(vref, 0, sizeof(double) * (size_t)(n + kWY) * n, c.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(tau, 0, sizeof(double) * (n + kWY), c.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(s->sacc, 0, sizeof(double) * 4, c.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(s->info, 0, sizeof(int) * 2, c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest_real: workspace reset");
  TriArgsR ta{n,     lda,
              G,     a,
              s->d,  s->e,
              s->e2, tau,
              vref,  reinterpret_cast<double*>(s->ybuf),
              reinterpret_cast<double*>(s->rnext), reinterpret_cast<double*>(s->rowcoef),
              vscale, s->sacc,
              s->bar, c.d_err, s->spart};
  void* args[] = {&ta};
  HPSI_LAUNCH(c, HPSI_K_TRIDIAG,
              (err = cudaLaunchCooperativeKernel(tri_kernel, dim3(G), dim3(df ? kDfThreads : kTriThreads), args, smem,
                                                 c.stream)));
  ++c.tri_calls;
  c.tri_flops += 4.0 / 3.0 * (double)n * (double)n * (double)n;
  if (err == cudaErrorCooperativeLaunchTooLarge) {
    cudaGetLastError();
    *fallback = true;
    return HPSI_OK;
  }
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest_real: tridiagonal reduction launch");
  // 2. eigenvalues, 3. eigenvectors of T (the same kernels as the complex solver)
  HPSI_LAUNCH(c, HPSI_K_EIGH,
              (k_eh_bisect<<<nwant, 32 * kBisWarps, 0, c.stream>>>(n, s->d, s->e, s->e2, nwant, s->lam)));
  rc = invit_all(c, *s, n, nwant, vec32 ? 2 : 3);
  if (rc) return rc;
  const double one = 1.0, zero = 0.0, mone = -1.0, mhalf = -0.5, three_half = 1.5;
  const size_t nz = (size_t)n * nwant;
  // float32 copies (vec32) live in the unused halves of the buffers sized for the complex solver:
  // Z and the Newton-Schulz output in Z2, the Gram matrix in gram, the reflectors and T factors
  // behind their float64 forms, the compact-WY products in w1 and w2
  float* zf = reinterpret_cast<float*>(s->Z2);
  float* vf = zf + nz;
  float* gf = reinterpret_cast<float*>(s->gram);
  // vec32: the float32 GEMMs below run as cuBLAS's float32 emulation on the bf16 tensor cores
  // (float32-accurate; finite operands, so without special-value passes), reset on every exit
  struct Emu {
    cublasHandle_t b = nullptr;
    void on(cublasHandle_t h) {
      b = h;
      cublasSetMathMode(h, CUBLAS_FP32_EMULATED_BF16X9_MATH);
      cublasSetEmulationStrategy(h, CUBLAS_EMULATION_STRATEGY_EAGER);
      cublasSetEmulationSpecialValuesSupport(h, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE);
    }
    ~Emu() {
      if (!b) return;
      cublasSetMathMode(b, CUBLAS_DEFAULT_MATH);
      cublasSetEmulationSpecialValuesSupport(b, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_DEFAULT);
    }
  } emu;
  if (vec32) emu.on(s->blas);
  if (vec32) {
    const float f1 = 1.f, f0 = 0.f, fmhalf = -0.5f, f3half = 1.5f;
    HPSI_LAUNCH(c, HPSI_K_EIGH, (k_eh_cvt<double, float><<<cvt_grid(nz), 256, 0, c.stream>>>(nz, s->Z, zf)));
    if (cublasSgemm(s->blas, CUBLAS_OP_T, CUBLAS_OP_N, nwant, nwant, n, &f1, zf, n, zf, n, &f0, gf, nwant) !=
        CUBLAS_STATUS_SUCCESS)
      return fail(c, HPSI_ECUDA, "eigh_lowest_real: Gram matrix of the eigenvectors failed");
    HPSI_LAUNCH(c, HPSI_K_EIGH,
                (k_eh_orthcheck<float><<<(nwant * nwant + 255) / 256, 256, 0, c.stream>>>(nwant, gf, 1e-4, s->info)));
    if (cudaMemcpyAsync(vf, zf, sizeof(float) * nz, cudaMemcpyDeviceToDevice, c.stream) != cudaSuccess ||
        cublasSgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, nwant, nwant, &fmhalf, zf, n, gf, nwant, &f3half, vf, n) !=
            CUBLAS_STATUS_SUCCESS)
      return fail(c, HPSI_ECUDA, "eigh_lowest_real: Newton-Schulz step failed");
  } else {
    if (cublasDgemm(s->blas, CUBLAS_OP_T, CUBLAS_OP_N, nwant, nwant, n, &one, s->Z, n, s->Z, n, &zero, s->gram,
                    nwant) != CUBLAS_STATUS_SUCCESS)
      return fail(c, HPSI_ECUDA, "eigh_lowest_real: Gram matrix of the eigenvectors failed");
    HPSI_LAUNCH(c, HPSI_K_EIGH,
                (k_eh_orthcheck<double><<<(nwant * nwant + 255) / 256, 256, 0, c.stream>>>(nwant, s->gram, 1e-4,
                                                                                          s->info)));
    // Newton-Schulz step straight into the output: v_out = Z (3 I - Z^T Z) / 2
    if (cudaMemcpyAsync(v_out, s->Z, sizeof(double) * nz, cudaMemcpyDeviceToDevice, c.stream) != cudaSuccess ||
        cublasDgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, n, nwant, nwant, &mhalf, s->Z, n, s->gram, nwant, &three_half,
                    v_out, n) != CUBLAS_STATUS_SUCCESS)
      return fail(c, HPSI_ECUDA, "eigh_lowest_real: Newton-Schulz step failed");
  }
  // 4. back-transformation, one compact-WY block of kWY reflectors at a time from the last
  if (n > 1) {
    if (df)
      HPSI_LAUNCH(c, HPSI_K_EIGH,
                  (k_eh_vscale_df<<<dim3((n + 255) / 256, n - 1), 256, 0, c.stream>>>(n, vscale, vref)));
    else
      HPSI_LAUNCH(c, HPSI_K_EIGH,
                  (k_eh_vscale_r<<<dim3((n + 255) / 256, n - 1), 256, 0, c.stream>>>(n, vscale, vref)));
    const int K = (n - 1 + kWY - 1) / kWY;
    if (cublasDgemmStridedBatched(s->blas, CUBLAS_OP_T, CUBLAS_OP_N, kWY, kWY, n - 1, &one, vref + 1, n,
                                  (long long)kWY * n, vref + 1, n, (long long)kWY * n, &zero, wgram, kWY,
                                  (long long)kWY * kWY, K) != CUBLAS_STATUS_SUCCESS)
      return fail(c, HPSI_ECUDA, "eigh_lowest_real: reflector Gram matrices failed");
    const size_t tsm = sizeof(double) * (size_t)kWY * (kWY - 1) / 2;
    if (df) HPSI_LAUNCH(c, HPSI_K_EIGH, (k_eh_tau_fix<<<(n - 1 + 255) / 256, 256, 0, c.stream>>>(n - 1, wgram, tau)));
    HPSI_LAUNCH(c, HPSI_K_EIGH, (k_eh_tfactor_r<<<dim3(kWY / 4, K), 128, tsm, c.stream>>>(wgram, tau, tfac)));
    if (vec32) {
      const size_t nv = (size_t)K * kWY * n, nt = (size_t)K * kWY * kWY;
      float* vr32 = reinterpret_cast<float*>(vref + (size_t)(n + kWY) * n);
      float* tf32 = reinterpret_cast<float*>(tfac + nt);
      float* w1f = reinterpret_cast<float*>(w1);
      float* w2f = reinterpret_cast<float*>(w2);
      HPSI_LAUNCH(c, HPSI_K_EIGH, (k_eh_cvt<double, float><<<cvt_grid(nv), 256, 0, c.stream>>>(nv, vref, vr32)));
      HPSI_LAUNCH(c, HPSI_K_EIGH, (k_eh_cvt<double, float><<<cvt_grid(nt), 256, 0, c.stream>>>(nt, tfac, tf32)));
      const float f1 = 1.f, f0 = 0.f, fm1 = -1.f;
      for (int k = K - 1; k >= 0; --k) {
        const int r0 = k * kWY + 1, m = n - r0;
        const float* V = vr32 + (size_t)k * kWY * n + r0;
        if (cublasSgemm(s->blas, CUBLAS_OP_T, CUBLAS_OP_N, kWY, nwant, m, &f1, V, n, vf + r0, n, &f0, w1f, kWY) !=
                CUBLAS_STATUS_SUCCESS ||
            cublasSgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, kWY, nwant, kWY, &f1, tf32 + (size_t)k * kWY * kWY, kWY,
                        w1f, kWY, &f0, w2f, kWY) != CUBLAS_STATUS_SUCCESS ||
            cublasSgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, m, nwant, kWY, &fm1, V, n, w2f, kWY, &f1, vf + r0, n) !=
                CUBLAS_STATUS_SUCCESS)
          return fail(c, HPSI_ECUDA, "eigh_lowest_real: back-transformation GEMM failed");
      }
    }
    for (int k = vec32 ? -1 : K - 1; k >= 0; --k) {
      const int r0 = k * kWY + 1, m = n - r0;
      double* V = vref + (size_t)k * kWY * n + r0;
      if (cublasDgemm(s->blas, CUBLAS_OP_T, CUBLAS_OP_N, kWY, nwant, m, &one, V, n, v_out + r0, n, &zero, w1, kWY) !=
              CUBLAS_STATUS_SUCCESS ||
          cublasDgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, kWY, nwant, kWY, &one, tfac + (size_t)k * kWY * kWY, kWY, w1,
                      kWY, &zero, w2, kWY) != CUBLAS_STATUS_SUCCESS ||
          cublasDgemm(s->blas, CUBLAS_OP_N, CUBLAS_OP_N, m, nwant, kWY, &mone, V, n, w2, kWY, &one, v_out + r0, n) !=
              CUBLAS_STATUS_SUCCESS)
        return fail(c, HPSI_ECUDA, "eigh_lowest_real: back-transformation GEMM failed");
    }
  }
  if (vec32) HPSI_LAUNCH(c, HPSI_K_EIGH, (k_eh_cvt<float, double><<<cvt_grid(nz), 256, 0, c.stream>>>(nz, vf, v_out)));
  err = cudaMemcpyAsync(w_out, s->lam, sizeof(double) * nwant, cudaMemcpyDeviceToDevice, c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest_real: eigenvalue copy");
  int info[2] = {0, 0};
  err = cudaMemcpyAsync(info, s->info, sizeof(int) * 2, cudaMemcpyDeviceToHost, c.stream);
  if (err != cudaSuccess) return cuda_fail(c, err, "eigh_lowest_real: status copy");
  rc = check_device_error(c);
  if (rc) return rc;
  ++c.eig_calls;
  if (info[0] != 0 || info[1] != 0) {
    *fallback = true;
    ++c.eig_fallbacks;
  }
  return HPSI_OK;
}

int eigh_reduced(Context& c, const double2* a, int lda, int n, int nwant, double* w_out, double2* v_out) {
  if (c.eigensolver == 1) {
    bool fallback = false;
    const int rc = eigh_lowest(c, a, lda, n, nwant, w_out, v_out, &fallback);
    if (rc || !fallback) return rc;
  }
  EighState* s = nullptr;
  const int rc = ensure_state(c, &s);
  if (rc) return rc;
  return eigh_zheevdx(c, *s, a, lda, n, nwant, w_out, v_out);
}

}  // namespace hpsi

extern "C" int hpsi_eigh_lowest(hpsi_ctx* ctx, int n, const void* a, int lda, int nwant, void* w_out, void* v_out) {
  if (!ctx) return HPSI_EINVAL;
  hpsi::Context& c = ctx->c;
  if (!a || !w_out || !v_out) return hpsi::fail(c, HPSI_EINVAL, "hpsi_eigh_lowest: null pointer");
  if (n < 1 || nwant < 1 || nwant > n || lda < n) return hpsi::fail(c, HPSI_EINVAL, "hpsi_eigh_lowest: bad sizes");
  return hpsi::eigh_reduced(c, static_cast<const double2*>(a), lda, n, nwant, static_cast<double*>(w_out),
                            static_cast<double2*>(v_out));
}

extern "C" int hpsi_eigh_lowest_sym(hpsi_ctx* ctx, int n, const void* a, int lda, int nwant, void* w_out,
                                    void* v_out) {
  if (!ctx) return HPSI_EINVAL;
  hpsi::Context& c = ctx->c;
  if (!a || !w_out || !v_out) return hpsi::fail(c, HPSI_EINVAL, "hpsi_eigh_lowest_sym: null pointer");
  if (n < 1 || nwant < 1 || nwant > n || lda < n) return hpsi::fail(c, HPSI_EINVAL, "hpsi_eigh_lowest_sym: bad sizes");
  if (c.eigensolver == 1) {
    bool fallback = false;
    const int rc = hpsi::eigh_lowest_real(c, static_cast<const double*>(a), lda, n, nwant, static_cast<double*>(w_out),
                                          static_cast<double*>(v_out), &fallback, false, c.eigh_df == 2);
    if (rc || !fallback) return rc;
  }
  return hpsi::fail(c, HPSI_EINVAL, "hpsi_eigh_lowest_sym: n too large for the library's real eigensolver");
}
