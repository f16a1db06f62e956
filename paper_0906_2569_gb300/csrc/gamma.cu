// Gamma-point real-wavefunction form (paper Sec. 4): at k = 0 the orbitals can be taken real, so
// psi(-G) = conj(psi(G)) and only the half sphere S+ is stored: G = 0 and, of every pair (G, -G),
// the member whose first nonzero Miller index is positive.  In the sphere's lexicographic order the
// entry npw-1-i is -G of entry i, so S+ is the last nh = (npw+1)/2 entries and G = 0 is entry
// i0 = nh-1 of the full list (entry 0 of the half list).
//
// H|psi> for real orbitals: two of them share one complex transform pair.  With f = psi_a + i psi_b
// (a complex function whose coefficients on the full sphere are f(G) = c_a(G) + i c_b(G) and
// f(-G) = conj(c_a(G)) + i conj(c_b(G))), F = H f gives
//     (H psi_a)(G) = (F(G) + conj(F(-G))) / 2,   (H psi_b)(G) = (F(G) - conj(F(-G))) / (2i),
// because H maps real functions to real ones (V is real; the projectors are checked at setup).
// So the complex operator of the library runs once per pair of bands, between a pack and an unpack
// kernel.
//
// Block Davidson on real orbitals (App. A.2.1 in the real basis of Sec. 4): a real orbital is the
// real vector x of length 2 nh with x = (c(0), 0) at G = 0 and x = sqrt2 (Re c(G), Im c(G)) for
// the other G of S+.  Then <a|b> = x_a . x_b, H is a real symmetric matrix in these coordinates,
// and every subspace product is a real GEMM with a quarter of the flops of the complex form.  The
// basis is float64 (HPSI_FP64) or float32 (HPSI_MIXED); residual norms, reduced matrices, their
// Cholesky factors and eigenproblems, and (mixed) the final Rayleigh quotients are float64.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "hpsi_internal.h"

namespace hpsi {

namespace {

constexpr double kSqrt2 = 1.4142135623730950488;
constexpr double kInvSqrt2 = 0.70710678118654752440;

template <typename T> struct V2;
template <> struct V2<double> { using type = double2; };
template <> struct V2<float> { using type = float2; };

__device__ __forceinline__ double2 ld2(const double2* p) { return *p; }
__device__ __forceinline__ void st2(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void st2(float2* p, double2 v) { *p = make_float2((float)v.x, (float)v.y); }

// Pack pairs of half-sphere bands into full-sphere complex bands: f[q] = x[2q] + i x[2q+1] (a
// missing odd partner is zero).  scaled: x holds the real-basis coordinates (sqrt2 c for G != 0).
template <typename S>
__global__ void k_gamma_pack(int npw, int nb, const S* __restrict__ x, int scaled, double2* __restrict__ f) {
  const int nh = (npw + 1) / 2, i0 = nh - 1;
  const int q = blockIdx.y;
  const int a = 2 * q, b = 2 * q + 1;
  const S* xa = x + (size_t)a * nh;
  const S* xb = x + (size_t)b * nh;
  double2* fq = f + (size_t)q * npw;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npw; i += gridDim.x * blockDim.x) {
    const bool neg = i < i0;
    const int h = neg ? i0 - i : i - i0;
    if constexpr (sizeof(S) == sizeof(float2)) {
      // float32 arithmetic (the float64 unit only widens the result)
      float2 ca = xa[h];
      float2 cb = b < nb ? xb[h] : make_float2(0.f, 0.f);
      if (scaled && h > 0) {
        ca.x *= (float)kInvSqrt2; ca.y *= (float)kInvSqrt2;
        cb.x *= (float)kInvSqrt2; cb.y *= (float)kInvSqrt2;
      }
      if (h == 0) {
        ca.y = 0.f;
        cb.y = 0.f;
      }
      if (neg) {
        ca.y = -ca.y;
        cb.y = -cb.y;
      }
      fq[i] = make_double2((double)(ca.x - cb.y), (double)(ca.y + cb.x));
    } else {
      double2 ca = ld2(xa + h);
      double2 cb = b < nb ? ld2(xb + h) : make_double2(0.0, 0.0);
      if (scaled && h > 0) {
        ca.x *= kInvSqrt2; ca.y *= kInvSqrt2;
        cb.x *= kInvSqrt2; cb.y *= kInvSqrt2;
      }
      if (h == 0) {   // a real orbital has a real G = 0 component
        ca.y = 0.0;
        cb.y = 0.0;
      }
      if (neg) {
        ca.y = -ca.y;
        cb.y = -cb.y;
      }
      fq[i] = make_double2(ca.x - cb.y, ca.y + cb.x);
    }
  }
}

// Unpack F = H f into the two bands' half-sphere results (see the file header), adding the
// nonlocal term given in real-basis coordinates: nl64 [nb][nr], or the float partial sums
// nl32 [ns32][nb][nr] (added in float64); neither: the local part alone.
template <typename S>
__global__ void k_gamma_unpack(int npw, int nb, const double2* __restrict__ F, int scaled,
                               const double* __restrict__ nl64, const float* __restrict__ nl32, int ns32,
                               S* __restrict__ y) {
  const int nh = (npw + 1) / 2, i0 = nh - 1;
  const size_t nr = 2 * (size_t)nh;
  const int q = blockIdx.y;
  const int a = 2 * q, b = 2 * q + 1;
  const double2* Fq = F + (size_t)q * npw;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
    if constexpr (sizeof(S) == sizeof(float2)) {
      // float32 result: float32 arithmetic, the float64 unit only narrows F and nl64
      const double2 fpd = Fq[i0 + h], fmd = Fq[i0 - h];
      const float2 fp = make_float2((float)fpd.x, (float)fpd.y), fm = make_float2((float)fmd.x, (float)fmd.y);
      float2 ya = make_float2(0.5f * (fp.x + fm.x), 0.5f * (fp.y - fm.y));
      float2 yb = make_float2(0.5f * (fp.y + fm.y), -0.5f * (fp.x - fm.x));
      if (scaled && h > 0) {
        ya.x *= (float)kSqrt2; ya.y *= (float)kSqrt2;
        yb.x *= (float)kSqrt2; yb.y *= (float)kSqrt2;
      }
      if (nl64 || nl32) {
        const float sn = (!scaled && h > 0) ? (float)kInvSqrt2 : 1.f;
        float na0 = 0.f, na1 = 0.f, nb0 = 0.f, nb1 = 0.f;
        const size_t ia = (size_t)a * nr + 2 * h, ib = (size_t)b * nr + 2 * h;
        if (nl64) {
          na0 = (float)nl64[ia];
          na1 = (float)nl64[ia + 1];
          if (b < nb) {
            nb0 = (float)nl64[ib];
            nb1 = (float)nl64[ib + 1];
          }
        } else {
          const size_t plane = (size_t)nb * nr;
          for (int sp = 0; sp < ns32; ++sp) {
            const float2 va = *reinterpret_cast<const float2*>(nl32 + sp * plane + ia);
            na0 += va.x;
            na1 += va.y;
            if (b < nb) {
              const float2 vb = *reinterpret_cast<const float2*>(nl32 + sp * plane + ib);
              nb0 += vb.x;
              nb1 += vb.y;
            }
          }
        }
        ya.x = fmaf(sn, na0, ya.x);
        ya.y = fmaf(sn, na1, ya.y);
        yb.x = fmaf(sn, nb0, yb.x);
        yb.y = fmaf(sn, nb1, yb.y);
      }
      y[(size_t)a * nh + h] = ya;
      if (b < nb) y[(size_t)b * nh + h] = yb;
      continue;
    }
    const double2 fp = Fq[i0 + h], fm = Fq[i0 - h];
    // conj(F(-G)) = (fm.x, -fm.y)
    double2 ya = make_double2(0.5 * (fp.x + fm.x), 0.5 * (fp.y - fm.y));
    double2 yb = make_double2(0.5 * (fp.y + fm.y), -0.5 * (fp.x - fm.x));
    if (scaled && h > 0) {
      ya.x *= kSqrt2; ya.y *= kSqrt2;
      yb.x *= kSqrt2; yb.y *= kSqrt2;
    }
    if (nl64 || nl32) {
      // the nonlocal term is in real-basis coordinates: 1/sqrt2 for coefficients at G != 0
      const double sn = (!scaled && h > 0) ? kInvSqrt2 : 1.0;
      double na0 = 0.0, na1 = 0.0, nb0 = 0.0, nb1 = 0.0;
      const size_t ia = (size_t)a * nr + 2 * h, ib = (size_t)b * nr + 2 * h;
      if (nl64) {
        na0 = nl64[ia];
        na1 = nl64[ia + 1];
        if (b < nb) {
          nb0 = nl64[ib];
          nb1 = nl64[ib + 1];
        }
      } else {
        const size_t plane = (size_t)nb * nr;
        for (int sp = 0; sp < ns32; ++sp) {
          const float2 va = *reinterpret_cast<const float2*>(nl32 + sp * plane + ia);
          na0 += (double)va.x;
          na1 += (double)va.y;
          if (b < nb) {
            const float2 vb = *reinterpret_cast<const float2*>(nl32 + sp * plane + ib);
            nb0 += (double)vb.x;
            nb1 += (double)vb.y;
          }
        }
      }
      ya.x = fma(sn, na0, ya.x);
      ya.y = fma(sn, na1, ya.y);
      yb.x = fma(sn, nb0, yb.x);
      yb.y = fma(sn, nb1, yb.y);
    }
    st2(y + (size_t)a * nh + h, ya);
    if (b < nb) st2(y + (size_t)b * nh + h, yb);
  }
}

// The projectors rephased by w_q = conj(sqrt(u_q)), so that beta'(-G) = conj(beta'(G)), in
// real-basis coordinates [P][2 nh].
__global__ void k_gamma_betar(int npw, const double2* __restrict__ beta, const double2* __restrict__ wph,
                              double* __restrict__ betar) {
  const int nh = (npw + 1) / 2, i0 = nh - 1;
  const int q = blockIdx.y;
  const double2 w = wph[q];
  const double2* bq = beta + (size_t)q * npw;
  double* out = betar + (size_t)q * 2 * nh;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
    const double2 b = bq[i0 + h];
    double re = w.x * b.x - w.y * b.y, im = w.x * b.y + w.y * b.x;
    if (h == 0) {
      im = 0.0;   // beta'(0) is real
    } else {
      re *= kSqrt2;
      im *= kSqrt2;
    }
    out[2 * h] = re;
    out[2 * h + 1] = im;
  }
}

// D'_pq = conj(w_p) D_pq w_q on D's CSR pattern (real when the Gamma form applies)
__global__ void k_gamma_dreal(int nproj, const int* __restrict__ rowptr, const int* __restrict__ col,
                              const double2* __restrict__ dval, const double2* __restrict__ wph,
                              double* __restrict__ dvalr) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nproj) return;
  const double2 wp = wph[p];
  for (int e = rowptr[p]; e < rowptr[p + 1]; ++e) {
    const double2 d = dval[e], wq = wph[col[e]];
    const double ax = wp.x * d.x + wp.y * d.y, ay = wp.x * d.y - wp.y * d.x;   // conj(w_p) D_pq
    dvalr[e] = ax * wq.x - ay * wq.y;
  }
}

int grid_x(size_t n) { return (int)std::min<size_t>(1024, (n + 255) / 256); }

// Build the rephased projectors and D' of problem p on first use (and their bf16 terms for a mixed
// context).
int gamma_nl_prepare(Context& c, Problem& p) {
  const int P = p.nproj;
  if (P == 0) return HPSI_OK;
  if (!p.d_betar) {
    if ((int)p.gamma_u.size() != P) return fail(c, HPSI_EINVAL, "Gamma-form projector phases are missing");
    std::vector<double2> w(P);
    for (int q = 0; q < P; ++q) {
      const double th = std::atan2(p.gamma_u[q].y, p.gamma_u[q].x);
      w[q] = make_double2(std::cos(0.5 * th), -std::sin(0.5 * th));
    }
    const int nr = 2 * ((p.npw + 1) / 2);
    double2* dw = nullptr;
    if (cudaMalloc((void**)&p.d_betar, sizeof(double) * (size_t)P * nr) != cudaSuccess ||
        cudaMalloc((void**)&p.d_dvalr, sizeof(double) * (size_t)std::max(1, p.nnz)) != cudaSuccess ||
        cudaMalloc((void**)&dw, sizeof(double2) * P) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(p.d_betar);
      cudaFree(p.d_dvalr);
      p.d_betar = nullptr;
      p.d_dvalr = nullptr;
      return fail(c, HPSI_ENOMEM, "device allocation of the Gamma-form projectors failed");
    }
    cudaError_t e = cudaMemcpyAsync(dw, w.data(), sizeof(double2) * P, cudaMemcpyHostToDevice, c.stream);
    if (e == cudaSuccess) {
      HPSI_LAUNCH(c, HPSI_K_GAMMA, (k_gamma_betar<<<dim3(grid_x((p.npw + 1) / 2), P), 256, 0, c.stream>>>(
                                       p.npw, p.d_beta, dw, p.d_betar)));
      if (p.nnz)
        HPSI_LAUNCH(c, HPSI_K_GAMMA, (k_gamma_dreal<<<(P + 127) / 128, 128, 0, c.stream>>>(
                                         P, p.d_rowptr, p.d_col, p.d_dval, dw, p.d_dvalr)));
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    }
    cudaFree(dw);
    if (e != cudaSuccess) {
      cudaFree(p.d_betar);
      cudaFree(p.d_dvalr);
      p.d_betar = nullptr;
      p.d_dvalr = nullptr;
      return cuda_fail(c, e, "Gamma-form projector setup");
    }
  }
  if (c.precision == HPSI_MIXED) {
    const int rc = gamma_prepare_tc(c, p);
    if (rc) return rc;
    return gamma_prepare_df(c, p);
  }
  return HPSI_OK;
}

}  // namespace

// y = H x for nb real orbitals in half-sphere storage (S = double2 or float2 elements, nh per
// band); scaled: real-basis coordinates in and out.  The local term runs on packed pairs of bands
// through the complex transforms; the nonlocal term runs on the real coordinates (half the work of
// the packed complex form) and is added while unpacking.  Counts nb band-applications.
template <typename S>
static int gamma_apply_t(Context& c, int ik, const S* x, S* y, int nb, bool scaled) {
  Problem& p = c.probs[ik];
  if (nb == 0) return HPSI_OK;
  constexpr int kMaxBlock = 65534;   // bands (and pairs) index gridDim.y
  if (nb > kMaxBlock) {
    const size_t nh = (size_t)(p.npw + 1) / 2;
    for (int b0 = 0; b0 < nb; b0 += kMaxBlock) {
      const int rc = gamma_apply_t<S>(c, ik, x + b0 * nh, y + b0 * nh, std::min(kMaxBlock, nb - b0), scaled);
      if (rc) return rc;
    }
    return HPSI_OK;
  }
  int rc = gamma_nl_prepare(c, p);
  if (rc) return rc;
  const int npairs = (nb + 1) / 2;
  const size_t bytes = sizeof(double2) * (size_t)npairs * p.npw;
  rc = ensure_buffer(c, &c.ws.gin, &c.ws.ginbytes, bytes);
  if (rc) return rc;
  rc = ensure_buffer(c, &c.ws.gout, &c.ws.goutbytes, bytes);
  if (rc) return rc;
  double2* f = static_cast<double2*>(c.ws.gin);
  double2* F = static_cast<double2*>(c.ws.gout);
  HPSI_LAUNCH(c, HPSI_K_GAMMA, (k_gamma_pack<S><<<dim3(grid_x(p.npw), npairs), 256, 0, c.stream>>>(
                                   p.npw, nb, x, scaled ? 1 : 0, f)));
  rc = local_apply(c, p, f, F, npairs);
  if (rc) return rc;
  const double* nl64 = nullptr;
  const float* nl32 = nullptr;
  int ns32 = 0;
  if (p.nproj > 0) {
    constexpr bool x32 = sizeof(S) == sizeof(float2);
    const int np = nl_prec(c);
    if (np == kNlProj64 && c.precision == HPSI_MIXED) {
      // projections to float64 accuracy (a double-float GEMM on the float32 pipes), add_vuspsi on
      // the tensor cores
      double* w = nullptr;
      rc = gamma_w_df(c, p, x, x32, nb, scaled, &w);
      if (!rc) rc = gamma_add_tc(c, p, w, nb, &nl32, &ns32);
    } else if (np == HPSI_FP64 || np == kNlProj64) {
      const int nr = 2 * ((p.npw + 1) / 2);
      rc = ensure_buffer(c, &c.ws.gnl, &c.ws.gnlbytes, sizeof(double) * (size_t)nb * nr);
      if (rc) return rc;
      double* out = static_cast<double*>(c.ws.gnl);
      rc = gamma_nonlocal_fp64(c, p, x, x32, nb, scaled, out);
      nl64 = out;
    } else {
      rc = gamma_nonlocal_mixed(c, p, x, x32, nb, scaled, &nl32, &ns32);
    }
    if (rc) return rc;
  }
  c.band_apps += nb;
  HPSI_LAUNCH(c, HPSI_K_GAMMA, (k_gamma_unpack<S><<<dim3(grid_x((p.npw + 1) / 2), npairs), 256, 0, c.stream>>>(
                                   p.npw, nb, F, scaled ? 1 : 0, nl64, nl32, ns32, y)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "gamma pack / unpack kernels");
  return HPSI_OK;
}

int gamma_apply(Context& c, int ik, const double2* x, double2* y, int nb, bool scaled) {
  return gamma_apply_t<double2>(c, ik, x, y, nb, scaled);
}

int gamma_check(Context& c, int ik, const char* who) {
  if (ik < 0 || ik >= (int)c.probs.size()) return fail(c, HPSI_EINVAL, std::string(who) + ": problem index out of range");
  const Problem& p = c.probs[ik];
  if (!p.gamma_ok) return fail(c, HPSI_EINVAL, std::string(who) + ": the Gamma-point real form does not apply: " + p.gamma_why);
  return HPSI_OK;
}

// ---------------------------------------------------------------------------------------------
// Block Davidson on real orbitals
// ---------------------------------------------------------------------------------------------

namespace {

constexpr double kDropAbs = 1e-8;   // overlap eigenvalues of unit corrections below this are dropped
constexpr double kCollapse = 1e-6;  // squared norm left after projection that marks a collapse
constexpr int kStall = 8;           // iterations without a 10% drop of the largest residual

template <typename T>
__device__ __forceinline__ double block_sum(double s, double* red) {
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[w] = s;
  __syncthreads();
  if (w == 0) {
    double r = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (lane == 0) red[32] = r;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

// Half-sphere complex128 coefficients -> real-basis coordinates (and back); one CTA row per band.
template <typename T>
__global__ void k_g_from_half(int nh, const double2* __restrict__ c, T* __restrict__ x) {
  const int b = blockIdx.y;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
    const double2 v = c[(size_t)b * nh + h];
    T* o = x + ((size_t)b * nh + h) * 2;
    if (h == 0) {
      o[0] = (T)v.x;
      o[1] = (T)0;
    } else {
      o[0] = (T)(kSqrt2 * v.x);
      o[1] = (T)(kSqrt2 * v.y);
    }
  }
}
// a = I (n x n, float64)
__global__ void k_g_eye(int n, double* __restrict__ a) {
  const size_t nn = (size_t)n * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x)
    a[i] = (i % n) == (i / n) ? 1.0 : 0.0;
}

template <typename T>
__global__ void k_g_to_half(int nh, const T* __restrict__ x, double2* __restrict__ c) {
  const int b = blockIdx.y;
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
    const T* v = x + ((size_t)b * nh + h) * 2;
    c[(size_t)b * nh + h] = h == 0 ? make_double2((double)v[0], 0.0)
                                   : make_double2(kInvSqrt2 * (double)v[0], kInvSqrt2 * (double)v[1]);
  }
}

// <G|H|G> of the full sphere -> both coordinates of each G of S+
template <typename T>
__global__ void k_g_hdiag(int nh, const double* __restrict__ hdiag, T* __restrict__ hd) {
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < nh; h += gridDim.x * blockDim.x) {
    const double v = hdiag[nh - 1 + h];
    hd[2 * h] = (T)v;
    hd[2 * h + 1] = (T)v;
  }
}

// Sum of squares of float32 values to float64 accuracy without a float64 instruction per element:
// each square split exactly by an FMA (q^2 = p + e) and accumulated in a (hi, lo) pair of floats
// through TwoSum; the _rn intrinsics keep the compiler from contracting or reassociating it.
struct SqAcc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float q) {
    const float p = __fmul_rn(q, q);
    const float e = __fmaf_rn(q, q, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// r_i = hx_i - eps_i x_i, stored in T, and ||r_i||_2 to float64 accuracy; one CTA per band.  A float32
// basis forms r in float32 with eps as a (hi, lo) pair of floats (two FMAs: r to within an ulp of
// itself), a float64 basis in float64.
template <typename T>
__global__ void __launch_bounds__(512) k_g_residual(int n, const T* __restrict__ x, const T* __restrict__ hx,
                                                    const double* __restrict__ eps, T* __restrict__ r,
                                                    double* __restrict__ rnorm) {
  __shared__ double red[33];
  const int b = blockIdx.x;
  const double e = eps[b];
  const T* xb = x + (size_t)b * n;
  const T* hb = hx + (size_t)b * n;
  T* rb = r + (size_t)b * n;
  double s = 0.0;
  if constexpr (sizeof(T) == 4) {
    const float eh = (float)e, el = (float)(e - (double)eh);
    SqAcc acc;
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
      const float xv = xb[g];
      const float q = __fmaf_rn(-el, xv, __fmaf_rn(-eh, xv, hb[g]));
      rb[g] = q;
      acc.add(q);
    }
    s = acc.value();
  } else {
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
      const T q = (T)((double)hb[g] - e * (double)xb[g]);
      rb[g] = q;
      s += (double)q * (double)q;
    }
  }
  s = block_sum<T>(s, red);
  if (threadIdx.x == 0) rnorm[b] = sqrt(s);
}

// t_j = r_{idx[j]} / clamp(hd - eps_{idx[j]}), normalised; one CTA per correction.  A preconditioner
// needs no exact quotient, and a float64 division is a long instruction sequence on this GPU: the
// float32 basis takes the quotient and its partial norms in float32, the float64 basis a float32
// reciprocal refined by one float64 Newton step (relative error ~1e-14).
template <typename T>
__global__ void __launch_bounds__(512) k_g_precondition(int n, const int* __restrict__ idx, const T* __restrict__ r,
                                                        const T* __restrict__ hd, const double* __restrict__ eps,
                                                        double tau, int eshift, T* __restrict__ t) {
  __shared__ double red[33];
  const int j = blockIdx.x, i = idx[j];
  const double e = eps[eshift >= 0 ? eshift : i];
  const T* rb = r + (size_t)i * n;
  T* tb = t + (size_t)j * n;
  double s = 0.0;
  if (sizeof(T) == 4) {
    const float ef = (float)e, tf = (float)tau;
    float sf = 0.f;
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
      float d = (float)hd[g] - ef;
      if (fabsf(d) < tf) d = d >= 0.f ? tf : -tf;
      const float q = (float)rb[g] * __frcp_rn(d);
      tb[g] = (T)q;
      sf = fmaf(q, q, sf);
    }
    s = sf;
  } else {
    for (int g = threadIdx.x; g < n; g += blockDim.x) {
      double d = (double)hd[g] - e;
      if (fabs(d) < tau) d = d >= 0.0 ? tau : -tau;
      double inv = (double)__frcp_rn((float)d);
      inv = fma(inv, fma(-d, inv, 1.0), inv);
      const T q = (T)((double)rb[g] * inv);
      tb[g] = q;
      s = fma((double)q, (double)q, s);
    }
  }
  s = block_sum<T>(s, red);
  const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  const T invT = (T)inv;
  for (int g = threadIdx.x; g < n; g += blockDim.x) tb[g] = tb[g] * invT;
}

template <typename T>
__global__ void __launch_bounds__(512) k_g_norm2(int n, const T* __restrict__ t, double* __restrict__ out) {
  __shared__ double red[33];
  const T* tb = t + (size_t)blockIdx.x * n;
  double s = 0.0;
  if constexpr (sizeof(T) == 4) {
    SqAcc acc;
    for (int g = threadIdx.x; g < n; g += blockDim.x) acc.add(tb[g]);
    s = acc.value();
  } else {
    for (int g = threadIdx.x; g < n; g += blockDim.x) s += (double)tb[g] * (double)tb[g];
  }
  s = block_sum<T>(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// t_j <- r_{idx[j]} / ||r_{idx[j]}|| for the listed j (corrections that collapsed into the basis)
template <typename T>
__global__ void k_g_fallback(int n, const int* __restrict__ which, const int* __restrict__ idx,
                             const T* __restrict__ r, const double* __restrict__ rnorm, T* __restrict__ t) {
  const int j = which[blockIdx.x], i = idx[j];
  const double s = 1.0 / rnorm[i];
  const T* rb = r + (size_t)i * n;
  T* tb = t + (size_t)j * n;
  for (int g = threadIdx.x; g < n; g += blockDim.x) tb[g] = (T)((double)rb[g] * s);
}

// float64 Rayleigh quotient and residual norm of each band: eps = x.hx / x.x, ||hx - eps x||
__global__ void __launch_bounds__(512) k_g_rayleigh(int n, const double* __restrict__ x, const double* __restrict__ hx,
                                                    double* __restrict__ eps, double* __restrict__ rnorm) {
  __shared__ double red[33];
  const int b = blockIdx.x;
  const double* xb = x + (size_t)b * n;
  const double* hb = hx + (size_t)b * n;
  double xx = 0.0, xh = 0.0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    xx = fma(xb[g], xb[g], xx);
    xh = fma(xb[g], hb[g], xh);
  }
  xx = block_sum<double>(xx, red);
  xh = block_sum<double>(xh, red);
  const double e = xh / xx;
  double rr = 0.0;
  for (int g = threadIdx.x; g < n; g += blockDim.x) {
    const double q = hb[g] - e * xb[g];
    rr = fma(q, q, rr);
  }
  rr = block_sum<double>(rr, red);
  if (threadIdx.x == 0) {
    eps[b] = e;
    rnorm[b] = sqrt(rr / xx);
  }
}

// dst (rows x cols, ldd) <- src (rows x cols, lds), converting the element type
template <typename A, typename B>
__global__ void k_g_copy(int rows, int cols, const A* __restrict__ src, int lds, B* __restrict__ dst, int ldd) {
  const size_t n = (size_t)rows * cols;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % rows), c = (int)(i / rows);
    dst[(size_t)c * ldd + r] = (B)src[(size_t)c * lds + r];
  }
}

// out[:, c] = V[:, first + c] / sqrt(w[first + c]) (canonical orthonormalisation), V ld n
template <typename T>
__global__ void k_g_canon(int n, int first, int nkeep, const double* __restrict__ v, const double* __restrict__ w,
                          T* __restrict__ out) {
  const size_t m = (size_t)n * nkeep;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % n), c = (int)(i / n);
    out[(size_t)c * n + r] = (T)(v[(size_t)(first + c) * n + r] / sqrt(w[first + c]));
  }
}

__global__ void k_g_diag(int n, const double* __restrict__ u, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = u[(size_t)i * n + i] * u[(size_t)i * n + i];
}

// rows perm[b] of src -> rows b of dst (n elements each)
template <typename T>
__global__ void k_g_gather(int n, const int* __restrict__ perm, const T* __restrict__ src, T* __restrict__ dst) {
  const T* s = src + (size_t)perm[blockIdx.x] * n;
  T* d = dst + (size_t)blockIdx.x * n;
  for (int g = threadIdx.x; g < n; g += blockDim.x) d[g] = s[g];
}

int grid_of(size_t n) { return (int)std::min<size_t>(4096, (n + 255) / 256); }   // grid-stride kernels

// cuBLAS by element type
cublasStatus_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, double alpha,
                    const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc) {
  return cublasDgemm(h, ta, tb, m, n, k, &alpha, A, lda, B, ldb, &beta, C, ldc);
}
cublasStatus_t gemm(cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k, double alpha,
                    const float* A, int lda, const float* B, int ldb, double beta, float* C, int ldc) {
  const float a = (float)alpha, b = (float)beta;
  return cublasSgemm(h, ta, tb, m, n, k, &a, A, lda, B, ldb, &b, C, ldc);
}
cublasStatus_t trsm_ru(cublasHandle_t h, int m, int n, const double* U, int ldu, double* B, int ldb) {
  const double one = 1.0;
  return cublasDtrsm(h, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, m, n, &one, U,
                     ldu, B, ldb);
}
cublasStatus_t trsm_ru(cublasHandle_t h, int m, int n, const float* U, int ldu, float* B, int ldb) {
  const float one = 1.f;
  return cublasStrsm(h, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, m, n, &one, U,
                     ldu, B, ldb);
}

}  // namespace

struct GamWork {
  int nh = 0, N = 0, mmax = 0, kmax = 0, prec = -1;
  void* phi = nullptr;     // T [mmax][n2]
  void* hphi = nullptr;    // T [mmax][n2]
  void* psi = nullptr;     // T [N][n2] Ritz vectors
  void* hpsi = nullptr;    // T [N][n2]
  void* r = nullptr;       // T [N][n2] residuals
  void* t = nullptr;       // T [max(N, kmax)][n2] scratch
  void* small = nullptr;   // T [mmax][kmax] reduced coefficients
  void* hcol = nullptr;    // T [mmax][kmax] columns of H_sub / overlaps in T
  void* hd = nullptr;      // T [n2] preconditioner diagonal
  double* hsub = nullptr;  // [mmax][mmax]
  double* evec = nullptr;  // [mmax][mmax]
  double* wv = nullptr;    // [mmax]
  double* ovl = nullptr;   // [kmax][kmax]
  double* eps = nullptr;   // [N]
  double* rnorm = nullptr; // [N]
  double* cn2 = nullptr;   // [max(N, kmax)]
  int* idx = nullptr;      // [N]
  int* idx2 = nullptr;     // [max(N, kmax)]
  int* info = nullptr;
  double* work = nullptr;  // cuSOLVER workspace
  int lwork = 0;
  double* x64 = nullptr;   // [N][n2] float64 Ritz vectors (mixed exit)
  double* hx64 = nullptr;  // [N][n2]
  double* rinv = nullptr;  // [nt][nt] product of inverse Cholesky factors (float32 basis)
};

struct GamHandles {
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t solver = nullptr;
  GamWork wk;
};

static void free_gwork(GamWork& w) {
  for (void* p : {w.phi, w.hphi, w.psi, w.hpsi, w.r, w.t, w.small, w.hcol, w.hd}) cudaFree(p);
  for (double* p : {w.hsub, w.evec, w.wv, w.ovl, w.eps, w.rnorm, w.cn2, w.work, w.x64, w.hx64, w.rinv}) cudaFree(p);
  cudaFree(w.idx);
  cudaFree(w.idx2);
  cudaFree(w.info);
  w = GamWork();
}

void gamma_release(Context& c) {
  GamHandles* h = reinterpret_cast<GamHandles*>(c.gam);
  if (!h) return;
  free_gwork(h->wk);
  if (h->blas) cublasDestroy(h->blas);
  if (h->solver) cusolverDnDestroy(h->solver);
  delete h;
  c.gam = nullptr;
}

#define GCK(x, what)                                      \
  do {                                                    \
    cudaError_t e_ = (x);                                 \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)
#define GBK(x, what)                                                                                   \
  do {                                                                                                 \
    int s_ = (int)(x);                                                                                 \
    if (s_ != 0) return fail(c, HPSI_ECUDA, std::string(what) + " failed with status " + std::to_string(s_)); \
  } while (0)

template <typename T>
class GammaDavidson {
 public:
  GammaDavidson(Context& c, GamHandles& h, int ik) : c_(c), h_(h), w_(h.wk), ik_(ik), p_(c.probs[ik]) {}

  int run(int N, double tol, int maxiter, double2* psio, double* eig_out, int* iters_out, double* resnorm_out);

 private:
  Context& c_;
  GamHandles& h_;
  GamWork& w_;
  int ik_;
  const Problem& p_;
  int n2_ = 0;

  T* phi() { return static_cast<T*>(w_.phi); }
  T* hphi() { return static_cast<T*>(w_.hphi); }
  T* psi() { return static_cast<T*>(w_.psi); }
  T* hpsi() { return static_cast<T*>(w_.hpsi); }
  T* res() { return static_cast<T*>(w_.r); }
  T* tmp() { return static_cast<T*>(w_.t); }
  T* small() { return static_cast<T*>(w_.small); }
  T* hcol() { return static_cast<T*>(w_.hcol); }

  int alloc(int N);
  int apply(const T* x, T* y, int nb) {
    using S = typename V2<T>::type;
    return gamma_apply_t<S>(c_, ik_, reinterpret_cast<const S*>(x), reinterpret_cast<S*>(y), nb, true);
  }
  int eig_lowest(const double* a, int lda, int n, int nwant);
  int chol(int n, double thr, bool relative, bool* ok);
  int overlap(const T* x, int n);
  int orth(const T* x, int n, T* out, int* nkeep, double thr, bool relative);
  int hsub_columns(int rows, int col0, int ncol);
};

template <typename T>
int GammaDavidson<T>::alloc(int N) {
  Context& c = c_;
  GamWork& w = w_;
  const int mmax = basis_of(c) * N, prec = sizeof(T) == 8 ? HPSI_FP64 : HPSI_MIXED;
  if (w.nh == (p_.npw + 1) / 2 && w.N == N && w.mmax == mmax && w.prec == prec) return HPSI_OK;
  free_gwork(w);
  w.nh = (p_.npw + 1) / 2;
  w.N = N;
  w.mmax = mmax;
  w.prec = prec;
  w.kmax = std::max(N, mmax / 2);
  const size_t n2 = 2 * (size_t)w.nh, v = sizeof(T) * n2, nt = std::max(N, w.kmax);
  auto al = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  bool ok = al(&w.phi, v * mmax) && al(&w.hphi, v * mmax) && al(&w.psi, v * N) && al(&w.hpsi, v * N) &&
            al(&w.r, v * N) && al(&w.t, v * nt) && al(&w.small, sizeof(T) * (size_t)mmax * w.kmax) &&
            al(&w.hcol, sizeof(T) * (size_t)mmax * w.kmax) && al(&w.hd, v) &&
            al((void**)&w.hsub, sizeof(double) * (size_t)mmax * mmax) &&
            al((void**)&w.evec, sizeof(double) * (size_t)mmax * mmax) && al((void**)&w.wv, sizeof(double) * mmax) &&
            al((void**)&w.ovl, sizeof(double) * nt * nt) && al((void**)&w.eps, sizeof(double) * N) &&
            al((void**)&w.rnorm, sizeof(double) * N) && al((void**)&w.cn2, sizeof(double) * nt) &&
            al((void**)&w.idx, sizeof(int) * N) && al((void**)&w.idx2, sizeof(int) * nt) &&
            al((void**)&w.info, sizeof(int));
  if (ok && prec == HPSI_MIXED)
    ok = al((void**)&w.x64, 8 * n2 * N) && al((void**)&w.hx64, 8 * n2 * N) &&
         al((void**)&w.rinv, sizeof(double) * nt * nt);
  if (!ok) {
    free_gwork(w);
    return fail(c, HPSI_ENOMEM, "davidson_solve_gamma: device allocation of the reduced basis failed");
  }
  int lw1 = 0, lw2 = 0, lw3 = 0;
  GBK(cusolverDnDsyevd_bufferSize(h_.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, mmax, w.evec, mmax,
                                  w.wv, &lw1),
      "cusolverDnDsyevd_bufferSize");
  int meig = 0;
  GBK(cusolverDnDsyevdx_bufferSize(h_.solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_UPPER,
                                   mmax, w.evec, mmax, 0.0, 0.0, 1, mmax, &meig, w.wv, &lw2),
      "cusolverDnDsyevdx_bufferSize");
  GBK(cusolverDnDpotrf_bufferSize(h_.solver, CUBLAS_FILL_MODE_UPPER, (int)nt, w.ovl, (int)nt, &lw3),
      "cusolverDnDpotrf_bufferSize");
  w.lwork = std::max(lw1, std::max(lw2, lw3));
  if (!al((void**)&w.work, sizeof(double) * (size_t)std::max(w.lwork, 1))) {
    free_gwork(w);
    return fail(c, HPSI_ENOMEM, "davidson_solve_gamma: workspace allocation failed");
  }
  return HPSI_OK;
}

// Lowest nwant eigenpairs of the symmetric leading n x n block of a (ld lda), float64: values in
// w.wv, vectors in the first nwant columns of w.evec (ld n).  The library's real eigensolver
// (HPSI_OPT_EIGENSOLVER = 1), cuSOLVER dsyevdx where it does not apply or hands the problem back.
// A float32 basis (HPSI_OPT_EIGH_DF >= 1) takes the vectors to float32 accuracy (they rotate
// float32 vectors) and the reduction in double-float arithmetic, the values to ~1e-13 relative.
template <typename T>
int GammaDavidson<T>::eig_lowest(const double* a, int lda, int n, int nwant) {
  Context& c = c_;
  GamWork& w = w_;
  if (c.eigensolver == 1) {
    bool fallback = false;
    const bool mixed = sizeof(T) == sizeof(float);
    const int rc = eigh_lowest_real(c, a, lda, n, nwant, w.wv, w.evec, &fallback, mixed && c.eigh_df >= 1,
                                    c.eigh_df == 2 || (mixed && c.eigh_df == 1));
    if (rc || !fallback) return rc;
  }
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_g_copy<double, double><<<grid_of((size_t)n * n), 256, 0, c.stream>>>(n, n, a, lda, w.evec, n)));
  int meig = 0;
  GBK(cusolverDnDsyevdx(h_.solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_UPPER, n, w.evec,
                        n, 0.0, 0.0, 1, nwant, &meig, w.wv, w.work, w.lwork, w.info),
      "cusolverDnDsyevdx");
  int info = 0;
  GCK(cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "info copy");
  GCK(cudaStreamSynchronize(c.stream), "reduced eigenproblem");
  if (info != 0 || meig < nwant)
    return fail(c, HPSI_ESINGULAR, "dsyevdx of the reduced matrix failed, info " + std::to_string(info));
  return HPSI_OK;
}

// Cholesky of the float64 matrix in w.ovl (n x n, ld n): ok if every squared pivot exceeds thr
// (relative to the largest when relative).
template <typename T>
int GammaDavidson<T>::chol(int n, double thr, bool relative, bool* ok) {
  Context& c = c_;
  GamWork& w = w_;
  *ok = false;
  GBK(cusolverDnDpotrf(h_.solver, CUBLAS_FILL_MODE_UPPER, n, w.ovl, n, w.work, w.lwork, w.info), "cusolverDnDpotrf");
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_g_diag<<<(n + 255) / 256, 256, 0, c.stream>>>(n, w.ovl, w.cn2)));
  int info = 0;
  std::vector<double> dg(n);
  GCK(cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "potrf info copy");
  GCK(cudaMemcpyAsync(dg.data(), w.cn2, sizeof(double) * n, cudaMemcpyDeviceToHost, c.stream), "potrf diag copy");
  GCK(cudaStreamSynchronize(c.stream), "potrf");
  if (info != 0) return HPSI_OK;
  double mx = 0.0, mn = 1e300;
  for (double v : dg) {
    mx = std::max(mx, v);
    mn = std::min(mn, v);
  }
  *ok = mn > (relative ? thr * mx : thr);
  return HPSI_OK;
}

// w.ovl = x^T x for the block x[0:n] (float64 copy of a T product)
template <typename T>
int GammaDavidson<T>::overlap(const T* x, int n) {
  Context& c = c_;
  GBK(gemm(h_.blas, CUBLAS_OP_T, CUBLAS_OP_N, n, n, n2_, 1.0, x, n2_, x, n2_, 0.0, hcol(), n), "gemm overlap");
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_g_copy<T, double><<<grid_of((size_t)n * n), 256, 0, c.stream>>>(n, n, hcol(), n, w_.ovl, n)));
  return HPSI_OK;
}

// Orthonormalise x[0:n] into out (no overlap with x): Cholesky QR, Cholesky QR twice for a
// moderately conditioned correction block, else canonically through the overlap's eigenvectors
// (directions with eigenvalue <= thr, relative to the largest if relative, are dropped).
template <typename T>
int GammaDavidson<T>::orth(const T* x, int n, T* out, int* nkeep, double thr, bool relative) {
  Context& c = c_;
  GamWork& w = w_;
  const bool f64 = sizeof(T) == 8;
  // A float64 basis: y <- y R^{-1} by TRSM with the factor in w.ovl.  A float32 basis: the product
  // M of the inverse factors is kept in float64 (w.rinv, M <- M R^{-1} by a small TRSM) and out = x M
  // is one float32 GEMM (emulated on the bf16 tensor cores by default), far cheaper than a float32
  // TRSM over the whole block; every pass still factors the Gram matrix of the vectors it produced.
  auto solve_with_factor = [&](T* y) -> int {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_g_copy<double, T><<<grid_of((size_t)n * n), 256, 0, c.stream>>>(n, n, w.ovl, n, hcol(), n)));
    GBK(trsm_ru(h_.blas, n2_, n, hcol(), n, y, n2_), "trsm");
    return HPSI_OK;
  };
  auto apply_inverse = [&](bool first) -> int {   // float32 basis: out = x M, M <- M R^{-1}
    if (first) HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_g_eye<<<grid_of((size_t)n * n), 256, 0, c.stream>>>(n, w.rinv)));
    const double one = 1.0;
    GBK(cublasDtrsm(h_.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, n, n, &one,
                    w.ovl, n, w.rinv, n),
        "trsm inverse factor");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_g_copy<double, T><<<grid_of((size_t)n * n), 256, 0, c.stream>>>(n, n, w.rinv, n, hcol(), n)));
    GBK(gemm(h_.blas, CUBLAS_OP_N, CUBLAS_OP_N, n2_, n, n, 1.0, x, n2_, hcol(), n, 0.0, out, n2_),
        "gemm orthonormalise");
    return HPSI_OK;
  };
  int rc = overlap(x, n);
  if (rc) return rc;
  bool ok = false;
  rc = chol(n, relative ? (f64 ? 1e-10 : 1e-6) : (f64 ? 1e-6 : 1e-2), relative, &ok);
  if (rc) return rc;
  if (ok) {
    *nkeep = n;
    if constexpr (sizeof(T) == 8) {
      GCK(cudaMemcpyAsync(out, x, sizeof(T) * (size_t)n * n2_, cudaMemcpyDeviceToDevice, c.stream), "copy");
      return solve_with_factor(out);
    } else {
      return apply_inverse(true);
    }
  }
  if (!relative) {
    rc = overlap(x, n);
    if (rc) return rc;
    rc = chol(n, 1e-6, false, &ok);
    if (rc) return rc;
    if (ok) {
      if (f64) {
        GCK(cudaMemcpyAsync(out, x, sizeof(T) * (size_t)n * n2_, cudaMemcpyDeviceToDevice, c.stream), "copy");
        rc = solve_with_factor(out);
      } else {
        rc = apply_inverse(true);
      }
      if (rc) return rc;
      rc = overlap(out, n);
      if (rc) return rc;
      rc = chol(n, 1e-2, false, &ok);
      if (rc) return rc;
      if (ok) {
        *nkeep = n;
        return f64 ? solve_with_factor(out) : apply_inverse(false);
      }
    }
  }
  rc = overlap(x, n);
  if (rc) return rc;
  rc = eig_lowest(w.ovl, n, n, n);
  if (rc) return rc;
  std::vector<double> lam(n);
  GCK(cudaMemcpyAsync(lam.data(), w.wv, sizeof(double) * n, cudaMemcpyDeviceToHost, c.stream), "overlap eigenvalues");
  GCK(cudaStreamSynchronize(c.stream), "overlap eigenvalues");
  const double cut = relative ? thr * lam[n - 1] : thr;
  int first = 0;
  while (first < n && !(lam[first] > cut && lam[first] > 1e-300)) ++first;
  const int nk = n - first;
  *nkeep = nk;
  if (nk == 0) return HPSI_OK;
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_g_canon<T><<<grid_of((size_t)n * nk), 256, 0, c.stream>>>(n, first, nk, w.evec, w.wv, small())));
  GBK(gemm(h_.blas, CUBLAS_OP_N, CUBLAS_OP_N, n2_, nk, n, 1.0, x, n2_, small(), n, 0.0, out, n2_),
      "gemm orthonormalise");
  return HPSI_OK;
}

// H_sub[0:rows, col0:col0+ncol] = phi[0:rows]^T hphi[col0:col0+ncol] (T product, stored in float64)
template <typename T>
int GammaDavidson<T>::hsub_columns(int rows, int col0, int ncol) {
  Context& c = c_;
  const int mmax = w_.mmax;
  GBK(gemm(h_.blas, CUBLAS_OP_T, CUBLAS_OP_N, rows, ncol, n2_, 1.0, phi(), n2_, hphi() + (size_t)col0 * n2_, n2_, 0.0,
           hcol(), mmax),
      "gemm H_sub columns");
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_g_copy<T, double><<<grid_of((size_t)rows * ncol), 256, 0, c.stream>>>(
                                      rows, ncol, hcol(), mmax, w_.hsub + (size_t)col0 * mmax, mmax)));
  return HPSI_OK;
}

template <typename T>
int GammaDavidson<T>::run(int N, double tol, int maxiter, double2* psio, double* eig_out, int* iters_out,
                          double* resnorm_out) {
  Context& c = c_;
  int rc = alloc(N);
  if (rc) return rc;
  GamWork& w = w_;
  const int nh = w.nh, mmax = w.mmax;
  n2_ = 2 * nh;
  const int n2 = n2_;
  const size_t vb = sizeof(T) * (size_t)n2;
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_g_hdiag<T><<<grid_of(nh), 256, 0, c.stream>>>(nh, p_.d_hdiag, static_cast<T*>(w.hd))));
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_g_from_half<T><<<dim3(grid_x(nh), N), 256, 0, c.stream>>>(nh, psio, tmp())));
  int nk = 0;
  rc = orth(tmp(), N, phi(), &nk, 1e-12, true);
  if (rc) return rc;
  if (nk < N) return fail(c, HPSI_EINVAL, "davidson_solve_gamma: initial guess is linearly dependent");
  rc = apply(phi(), hphi(), N);
  if (rc) return rc;
  int m = N;
  rc = hsub_columns(m, 0, m);
  if (rc) return rc;
  std::vector<double> rn(N), ev(N);
  std::vector<int> uidx(N), asel;
  int it = 0;
  bool converged = false, thick = c.thick_restart != 0, refresh = false;
  int stall = 0;
  double best = INFINITY;
  auto restart_size = [&](int m_avail) { return thick ? std::min(m_avail, std::min(w.kmax, std::max(N, mmax / 2))) : N; };
  for (;;) {
    const int nev = m + N > mmax ? std::max(N, restart_size(m)) : N;
    rc = eig_lowest(w.hsub, mmax, m, nev);
    if (rc) return rc;
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_g_copy<double, T><<<grid_of((size_t)m * N), 256, 0, c.stream>>>(m, N, w.evec, m, small(), m)));
    GBK(gemm(h_.blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, N, m, 1.0, phi(), n2, small(), m, 0.0, psi(), n2), "gemm Ritz");
    GBK(gemm(h_.blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, N, m, 1.0, hphi(), n2, small(), m, 0.0, hpsi(), n2),
        "gemm H Ritz");
    GCK(cudaMemcpyAsync(w.eps, w.wv, sizeof(double) * N, cudaMemcpyDeviceToDevice, c.stream), "eps copy");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_g_residual<T><<<N, 512, 0, c.stream>>>(n2, psi(), hpsi(), w.eps, res(), w.rnorm)));
    GCK(cudaMemcpyAsync(rn.data(), w.rnorm, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream), "norm copy");
    GCK(cudaMemcpyAsync(ev.data(), w.eps, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream), "eig copy");
    GCK(cudaStreamSynchronize(c.stream), "davidson iteration");
    rc = check_device_error(c);
    if (rc) return rc;
    int nc = 0;
    double rmax = 0.0;
    for (int i = 0; i < N; ++i) {
      rmax = std::max(rmax, rn[i]);
      if (!(rn[i] <= tol)) uidx[nc++] = i;
    }
    if (nc == 0) {
      converged = true;
      break;
    }
    if (it >= maxiter) break;
    ++it;
    if (rmax < 0.9 * best) {
      best = rmax;
      stall = 0;
    } else if (++stall >= kStall) {
      stall = 0;
      if (thick) thick = false;
      else refresh = true;
    }
    if (m + nc > mmax || refresh) {
      const int keep = refresh ? N : restart_size(m);
      if (keep <= N) {
        GCK(cudaMemcpyAsync(phi(), psi(), vb * keep, cudaMemcpyDeviceToDevice, c.stream), "restart copy");
        GCK(cudaMemcpyAsync(hphi(), hpsi(), vb * keep, cudaMemcpyDeviceToDevice, c.stream), "restart copy");
      } else {
        if (keep > nev) {
          rc = eig_lowest(w.hsub, mmax, m, keep);
          if (rc) return rc;
        }
        HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                    (k_g_copy<double, T><<<grid_of((size_t)m * keep), 256, 0, c.stream>>>(m, keep, w.evec, m, small(), m)));
        for (int pass = 0; pass < 2; ++pass) {
          T* src = pass == 0 ? phi() : hphi();
          GBK(gemm(h_.blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, keep, m, 1.0, src, n2, small(), m, 0.0, tmp(), n2),
              "gemm restart");
          GCK(cudaMemcpyAsync(src, tmp(), vb * keep, cudaMemcpyDeviceToDevice, c.stream), "restart copy");
        }
      }
      if (refresh) {
        rc = apply(phi(), hphi(), keep);
        if (rc) return rc;
        refresh = false;
      }
      m = keep;
      rc = hsub_columns(m, 0, m);
      if (rc) return rc;
    }
    GCK(cudaMemcpyAsync(w.idx, uidx.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, c.stream), "index copy");
    T* tnew = phi() + (size_t)m * n2;
    const int eshift = c.opt_shift == 1 ? N - 1 : -1;
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_g_precondition<T><<<nc, 512, 0, c.stream>>>(
                                        n2, w.idx, res(), static_cast<const T*>(w.hd), w.eps, c.opt_tau, eshift, tnew)));
    // block Gram-Schmidt against phi[0:m], twice; corrections that lie in the basis are replaced
    // by their raw residuals (orthogonal to the basis by the Galerkin condition)
    auto project = [&]() -> int {
      GBK(gemm(h_.blas, CUBLAS_OP_T, CUBLAS_OP_N, m, nc, n2, 1.0, phi(), n2, tnew, n2, 0.0, small(), m),
          "gemm projection");
      GBK(gemm(h_.blas, CUBLAS_OP_N, CUBLAS_OP_N, n2, nc, m, -1.0, phi(), n2, small(), m, 1.0, tnew, n2),
          "gemm projection update");
      return HPSI_OK;
    };
    for (int round = 0; round < 2; ++round) {
      if ((rc = project()) || (rc = project())) return rc;
      if (round == 1) break;
      std::vector<double> cn(nc);
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_g_norm2<T><<<nc, 512, 0, c.stream>>>(n2, tnew, w.cn2)));
      GCK(cudaMemcpyAsync(cn.data(), w.cn2, sizeof(double) * nc, cudaMemcpyDeviceToHost, c.stream), "norm copy");
      GCK(cudaStreamSynchronize(c.stream), "correction norms");
      std::vector<int> col;
      for (int j = 0; j < nc; ++j)
        if (!(cn[j] >= kCollapse)) col.push_back(j);
      if (col.empty()) break;
      GCK(cudaMemcpyAsync(w.idx2, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice, c.stream),
          "index copy");
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                  (k_g_fallback<T><<<(int)col.size(), 256, 0, c.stream>>>(n2, w.idx2, w.idx, res(), w.rnorm, tnew)));
    }
    int nkeep = 0;
    rc = orth(tnew, nc, tmp(), &nkeep, kDropAbs, false);
    if (rc) return rc;
    if (nkeep == 0) {
      converged = rmax <= tol;
      break;
    }
    GCK(cudaMemcpyAsync(tnew, tmp(), vb * nkeep, cudaMemcpyDeviceToDevice, c.stream), "basis copy");
    rc = apply(tnew, hphi() + (size_t)m * n2, nkeep);
    if (rc) return rc;
    rc = hsub_columns(m + nkeep, m, nkeep);
    if (rc) return rc;
    m += nkeep;
  }
  // Output.  float64: the Ritz pairs of the last step.  float32 basis: Rayleigh quotients in
  // float64 with one more application of H (float64 unless HPSI_OPT_FINAL_FP64 is 0), sorted.
  std::vector<int> perm(N);
  for (int i = 0; i < N; ++i) perm[i] = i;
  if (sizeof(T) == 8) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_g_to_half<T><<<dim3(grid_x(nh), N), 256, 0, c.stream>>>(nh, psi(), psio)));
  } else {
    const size_t n = (size_t)N * n2;
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_g_copy<T, double><<<grid_of(n), 256, 0, c.stream>>>((int)n2, N, psi(), n2, w.x64, n2)));
    final_precision_begin(c);
    rc = gamma_apply_t<double2>(c, ik_, reinterpret_cast<const double2*>(w.x64), reinterpret_cast<double2*>(w.hx64),
                                N, true);
    final_precision_end(c);
    if (rc) return rc;
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_g_rayleigh<<<N, 512, 0, c.stream>>>(n2, w.x64, w.hx64, w.eps, w.rnorm)));
    GCK(cudaMemcpyAsync(ev.data(), w.eps, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream), "eig copy");
    GCK(cudaMemcpyAsync(rn.data(), w.rnorm, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream), "norm copy");
    GCK(cudaStreamSynchronize(c.stream), "davidson end");
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return ev[a] < ev[b]; });
    GCK(cudaMemcpyAsync(w.idx, perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice, c.stream), "perm copy");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_g_gather<double><<<N, 256, 0, c.stream>>>(n2, w.idx, w.x64, w.hx64)));
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_g_to_half<double><<<dim3(grid_x(nh), N), 256, 0, c.stream>>>(nh, w.hx64, psio)));
  }
  GCK(cudaStreamSynchronize(c.stream), "davidson end");
  rc = check_device_error(c);
  if (rc) return rc;
  for (int i = 0; i < N; ++i) {
    eig_out[i] = ev[perm[i]];
    if (resnorm_out) resnorm_out[i] = rn[perm[i]];
  }
  if (iters_out) *iters_out = it;
  if (!converged) return fail(c, HPSI_ENOTCONV, "davidson_solve_gamma: not converged within maxiter");
  return HPSI_OK;
}

int gamma_davidson_run(Context& c, int ik, int nbnd, double tol, int maxiter, double2* psio, double* eig_out,
                       int* iters_out, double* resnorm_out) {
  GamHandles* h = reinterpret_cast<GamHandles*>(c.gam);
  if (!h) {
    h = new GamHandles();
    c.gam = h;
    GBK(cublasCreate(&h->blas), "cublasCreate");
    GBK(cusolverDnCreate(&h->solver), "cusolverDnCreate");
  }
  GBK(cublasSetStream(h->blas, c.stream), "cublasSetStream");
  GBK(cusolverDnSetStream(h->solver, c.stream), "cusolverDnSetStream");
  if (c.precision == HPSI_MIXED) {
    // HPSI_OPT_GAMMA_GEMM = 1 (default): the float32 subspace GEMMs emulated by cuBLAS with bf16
    // tensor-core products (float32-accurate); 0: float32 on the CUDA cores
    const bool emu = c.gamma_gemm == 1;
    GBK(cublasSetMathMode(h->blas, emu ? CUBLAS_FP32_EMULATED_BF16X9_MATH : CUBLAS_DEFAULT_MATH), "cublasSetMathMode");
    if (emu) {
      GBK(cublasSetEmulationStrategy(h->blas, CUBLAS_EMULATION_STRATEGY_EAGER), "cublasSetEmulationStrategy");
      // the basis and its products are finite (a NaN would surface in the float64 residual norms),
      // so the emulation needs no infinity / NaN patching passes over its operands
      GBK(cublasSetEmulationSpecialValuesSupport(h->blas, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE),
          "cublasSetEmulationSpecialValuesSupport");
    }
    GammaDavidson<float> d(c, *h, ik);
    const int rc = d.run(nbnd, tol, maxiter, psio, eig_out, iters_out, resnorm_out);
    cublasSetMathMode(h->blas, CUBLAS_DEFAULT_MATH);
    cublasSetEmulationSpecialValuesSupport(h->blas, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_DEFAULT);
    return rc;
  }
  GammaDavidson<double> d(c, *h, ik);
  return d.run(nbnd, tol, maxiter, psio, eig_out, iters_out, resnorm_out);
}

}  // namespace hpsi

using namespace hpsi;

extern "C" int hpsi_apply_gamma(hpsi_ctx* ctx, int ik, const void* psi_in, void* hpsi_out, int nbnd) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  int rc = gamma_check(c, ik, "hpsi_apply_gamma");
  if (rc) return rc;
  if (nbnd < 0) return fail(c, HPSI_EINVAL, "hpsi_apply_gamma: nbnd < 0");
  if (nbnd == 0) return HPSI_OK;
  if (!psi_in || !hpsi_out) return fail(c, HPSI_EINVAL, "hpsi_apply_gamma: null pointer");
  const Problem& p = c.probs[ik];
  const size_t bytes = sizeof(double2) * (size_t)nbnd * ((p.npw + 1) / 2);
  const char* a0 = static_cast<const char*>(psi_in);
  const char* b0 = static_cast<const char*>(hpsi_out);
  if (a0 < b0 + bytes && b0 < a0 + bytes) return fail(c, HPSI_EINVAL, "hpsi_apply_gamma: psi_in and hpsi_out overlap");
  const int ka = pointer_kind(psi_in), kb = pointer_kind(hpsi_out);
  if (ka < 0 || kb < 0 || ka != kb)
    return fail(c, HPSI_EINVAL, "hpsi_apply_gamma: psi_in and hpsi_out must both be device or both be host memory");
  if (ka == 1)
    return gamma_apply(c, ik, static_cast<const double2*>(psi_in), static_cast<double2*>(hpsi_out), nbnd, false);
  rc = ensure_buffer(c, &c.ws.stage_in, &c.ws.stage_in_bytes, bytes);
  if (rc) return rc;
  rc = ensure_buffer(c, &c.ws.stage_out, &c.ws.stage_out_bytes, bytes);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(c.ws.stage_in, psi_in, bytes, cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "hpsi_apply_gamma host->device copy");
  rc = gamma_apply(c, ik, static_cast<const double2*>(c.ws.stage_in), static_cast<double2*>(c.ws.stage_out), nbnd,
                   false);
  if (rc) return rc;
  e = cudaMemcpyAsync(hpsi_out, c.ws.stage_out, bytes, cudaMemcpyDeviceToHost, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "hpsi_apply_gamma device->host copy");
  return check_device_error(c);
}

extern "C" int davidson_solve_gamma(hpsi_ctx* ctx, int ik, int nbnd, double tol, int maxiter, void* psi_inout,
                                    double* eig_out, int* iters_out, double* resnorm_out) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  int rc = gamma_check(c, ik, "davidson_solve_gamma");
  if (rc) return rc;
  const Problem& p = c.probs[ik];
  if (nbnd < 1 || (long long)nbnd * basis_of(c) > p.npw)
    return fail(c, HPSI_EINVAL, "davidson_solve_gamma: nbnd times the basis factor must not exceed npw");
  if (!(tol > 0.0) || maxiter < 1 || !psi_inout || !eig_out)
    return fail(c, HPSI_EINVAL, "davidson_solve_gamma: bad argument");
  const int kind = pointer_kind(psi_inout);
  if (kind < 0) return fail(c, HPSI_EINVAL, "davidson_solve_gamma: psi_inout is not a valid pointer");
  const size_t bytes = sizeof(double2) * (size_t)nbnd * ((p.npw + 1) / 2);
  double2* dpsi = static_cast<double2*>(psi_inout);
  if (kind == 0) {
    rc = ensure_buffer(c, &c.ws.stage_in, &c.ws.stage_in_bytes, bytes);
    if (rc) return rc;
    dpsi = static_cast<double2*>(c.ws.stage_in);
    cudaError_t e = cudaMemcpyAsync(dpsi, psi_inout, bytes, cudaMemcpyHostToDevice, c.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "davidson_solve_gamma host->device copy");
  }
  rc = gamma_davidson_run(c, ik, nbnd, tol, maxiter, dpsi, eig_out, iters_out, resnorm_out);
  if (kind == 0 && (rc == HPSI_OK || rc == HPSI_ENOTCONV)) {
    cudaError_t e = cudaMemcpyAsync(psi_inout, dpsi, bytes, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "davidson_solve_gamma device->host copy");
  }
  return rc;
}
