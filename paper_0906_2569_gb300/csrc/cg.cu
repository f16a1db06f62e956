// Band-by-band preconditioned conjugate-gradient eigensolver (paper App. A.2.2), on one GPU.
//
// Band i minimises <psi|H|psi> over unit vectors orthogonal to the bands j < i found before it.
// The paper writes the minimisation on y = P^-1 psi with H~ = P H P, S~ = P S P (S = I here) and
// notes that only P g, P h and P^2 are needed; on psi = P y one step is
//   lambda = <psi|P^2 H|psi> / <psi|P^2|psi>      (makes the gradient S~-orthogonal to y)
//   P g    = P^2 (H psi - lambda psi), minus its components along the bands j < i
//   P h    = P g + gamma P h_prev,  gamma = <P g - P g_prev|P g> / <P g_prev|P g_prev>  (Polak-Ribiere)
//   P h   -= psi <psi|P h>,  P n = P h / ||P h||
//   psi   <- psi cos(theta) + P n sin(theta),  theta = atan(a / (eps - b)) / 2 at the minimum,
//            a = 2 Re<psi|H|P n>, b = <P n|H|P n>, eps = <psi|H|psi>
// with the kinetic-only P^2 = 1 / max(|k+G|^2 / 2, t_min) (the paper's 2m / (hbar^2 |k+G|^2) in
// Hartree units, floored where it is undefined at k + G = 0).  H psi is carried along the rotation,
// so every step costs one application of H to one band.
//
// GPU layout: psi and the bands are the caller's [nbnd][npw] complex128 rows; the vectors of the
// current band (H psi, P g, P g_prev, P h, P n, H P n) live in one work block.  The reductions and
// the scalar algebra of a step run in three single-CTA kernels (1024 threads, float64 sums); the
// scalars stay on the device, and the host reads one residual norm per step for the stopping test.
// The Gram-Schmidt against the lower bands is two cuBLAS ZGEMV pairs.
#include <cublas_v2.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "hpsi_internal.h"

namespace hpsi {

namespace {

constexpr int kCgThreads = 1024;
constexpr double kPi = 3.14159265358979323846;

struct CgScalars {
  double eps, res2, lam;
  double gg, gg_prev;
  double hn2;     // ||P h||^2 of the step's direction
  double n0;      // squared norm of the band's start vector after the Gram-Schmidt
  double a, b, theta;
  int first;   // 1 on the first step of a band: no conjugation
};

struct CgState {
  cublasHandle_t blas = nullptr;
  int npw = 0, nbnd = 0;
  double2* work = nullptr;     // [6][npw]: hpsi, pg, pg_prev, ph, pn, hpn
  double2* coef = nullptr;     // [nbnd] Gram-Schmidt coefficients
  double* p2 = nullptr;        // [npw]
  CgScalars* sc = nullptr;
  int p2_ik = -1;
  double p2_tmin = -1.0;
};

// Sum of K doubles over the block; every thread receives the totals in v.
template <int K>
__device__ void block_sums(double (&v)[K]) {
  __shared__ double red[K][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[k][wid] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double x = lane < nw ? red[k][lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    v[k] = x;
  }
  __syncthreads();
}

__device__ __forceinline__ double re_dot(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }   // Re(conj(a) b)

__global__ void k_cg_p2(int npw, const double* __restrict__ kin, double tmin, double* __restrict__ p2) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < npw) p2[g] = 1.0 / fmax(kin[g], tmin);
}

// psi /= ||psi|| (the squared norm goes to sc->n0); single CTA.
__global__ void __launch_bounds__(kCgThreads) k_cg_normalize(int npw, double2* __restrict__ psi,
                                                             CgScalars* __restrict__ sc) {
  double v[1] = {0.0};
  for (int g = threadIdx.x; g < npw; g += blockDim.x) v[0] += re_dot(psi[g], psi[g]);
  block_sums<1>(v);
  const double s = v[0] > 0.0 ? 1.0 / sqrt(v[0]) : 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) psi[g] = make_double2(psi[g].x * s, psi[g].y * s);
  if (threadIdx.x == 0) {
    sc->n0 = v[0];
    sc->first = 1;
  }
}

// eps = <psi|H psi> / <psi|psi>, lambda = <psi|P^2 H psi> / <psi|P^2 psi>; then, in a second pass,
// ||H psi - eps psi||^2 and P g = P^2 (H psi - lambda psi).  Single CTA.
__global__ void __launch_bounds__(kCgThreads) k_cg_state(int npw, const double2* __restrict__ psi,
                                                         const double2* __restrict__ hpsi,
                                                         const double* __restrict__ p2, double2* __restrict__ pg,
                                                         CgScalars* __restrict__ sc) {
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 x = psi[g], hx = hpsi[g];
    const double w = p2[g], e = re_dot(x, hx);
    v[0] += e;
    v[1] += re_dot(x, x);
    v[2] += w * e;
    v[3] += w * re_dot(x, x);
  }
  block_sums<4>(v);
  const double eps = v[0] / v[1], lam = v[2] / v[3];
  double r[1] = {0.0};
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 x = psi[g], hx = hpsi[g];
    const double2 d = make_double2(hx.x - eps * x.x, hx.y - eps * x.y);
    r[0] += re_dot(d, d);
    const double w = p2[g];
    pg[g] = make_double2(w * (hx.x - lam * x.x), w * (hx.y - lam * x.y));
  }
  block_sums<1>(r);
  if (threadIdx.x == 0) {
    sc->eps = eps;
    sc->lam = lam;
    sc->res2 = r[0];
  }
}

// Polak-Ribiere direction from P g (already orthogonal to the lower bands): P h = P g + gamma P h,
// re-orthogonalised to psi and normalised into P n; P g is kept as P g_prev.  Single CTA.
__global__ void __launch_bounds__(kCgThreads) k_cg_direction(int npw, const double2* __restrict__ psi,
                                                             const double2* __restrict__ pg,
                                                             double2* __restrict__ pg_prev, double2* __restrict__ ph,
                                                             double2* __restrict__ pn, CgScalars* __restrict__ sc) {
  const bool first = sc->first != 0;
  double v[2] = {0.0, 0.0};
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 x = pg[g];
    v[0] += re_dot(x, x);
    if (!first) v[1] += re_dot(pg_prev[g], x);
  }
  block_sums<2>(v);
  const double gg = v[0];
  const double gamma = first ? 0.0 : (gg - v[1]) / sc->gg_prev;
  double z[2] = {0.0, 0.0};   // <psi|P h>
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 x = pg[g];
    const double2 h = first ? x : make_double2(x.x + gamma * ph[g].x, x.y + gamma * ph[g].y);
    ph[g] = h;
    const double2 p = psi[g];
    z[0] += p.x * h.x + p.y * h.y;
    z[1] += p.x * h.y - p.y * h.x;
  }
  block_sums<2>(z);
  double n[1] = {0.0};
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 p = psi[g], h0 = ph[g];
    const double2 h = make_double2(h0.x - (p.x * z[0] - p.y * z[1]), h0.y - (p.x * z[1] + p.y * z[0]));
    ph[g] = h;
    n[0] += re_dot(h, h);
  }
  block_sums<1>(n);
  const double s = n[0] > 0.0 ? 1.0 / sqrt(n[0]) : 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 h = ph[g];
    pn[g] = make_double2(h.x * s, h.y * s);
    pg_prev[g] = pg[g];
  }
  if (threadIdx.x == 0) {
    sc->gg_prev = gg;
    sc->gg = gg;
    sc->hn2 = n[0];
    sc->first = 0;
  }
}

// The exact minimum of <psi|H|psi> on psi cos t + P n sin t, then the rotation of psi and H psi.
// Single CTA.
__global__ void __launch_bounds__(kCgThreads) k_cg_move(int npw, double2* __restrict__ psi, double2* __restrict__ hpsi,
                                                        const double2* __restrict__ pn,
                                                        const double2* __restrict__ hpn, CgScalars* __restrict__ sc) {
  double v[2] = {0.0, 0.0};
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 hn = hpn[g];
    v[0] += re_dot(psi[g], hn);
    v[1] += re_dot(pn[g], hn);
  }
  block_sums<2>(v);
  const double eps = sc->eps, a = 2.0 * v[0], b = v[1];
  // stationary angles of E(t) = eps cos^2 t + b sin^2 t + a sin t cos t: t0 and t0 + pi/2
  const double t0 = eps != b ? 0.5 * atan(a / (eps - b)) : (a >= 0.0 ? 0.25 : -0.25) * kPi;
  const double t1 = t0 + 0.5 * kPi;
  auto energy = [&](double t) {
    const double cs = cos(t), sn = sin(t);
    return eps * cs * cs + b * sn * sn + a * sn * cs;
  };
  // a zero direction (nothing left to minimise along) leaves psi where it is
  const double t = !(sc->hn2 > 0.0) ? 0.0 : (energy(t1) < energy(t0) ? t1 : t0);
  const double cs = cos(t), sn = sin(t);
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 x = psi[g], n = pn[g], hx = hpsi[g], hn = hpn[g];
    psi[g] = make_double2(cs * x.x + sn * n.x, cs * x.y + sn * n.y);
    hpsi[g] = make_double2(cs * hx.x + sn * hn.x, cs * hx.y + sn * hn.y);
  }
  if (threadIdx.x == 0) {
    sc->a = a;
    sc->b = b;
    sc->theta = t;
  }
}

#define CCK(x, what)                                      \
  do {                                                    \
    cudaError_t e_ = (x);                                 \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)
#define CBK(x, what)                                                                              \
  do {                                                                                            \
    if ((x) != CUBLAS_STATUS_SUCCESS) return fail(c, HPSI_ECUDA, std::string("cg_solve: ") + what); \
  } while (0)

int ensure_cg(Context& c, int npw, int nbnd, CgState** out) {
  CgState* s = reinterpret_cast<CgState*>(c.cg);
  if (!s) {
    s = new CgState();
    c.cg = s;
    if (cublasCreate(&s->blas) != CUBLAS_STATUS_SUCCESS) return fail(c, HPSI_ECUDA, "cg_solve: cublasCreate");
  }
  if (cublasSetStream(s->blas, c.stream) != CUBLAS_STATUS_SUCCESS) return fail(c, HPSI_ECUDA, "cg_solve: cublasSetStream");
  if (npw > s->npw || nbnd > s->nbnd || !s->sc) {
    cudaFree(s->work);
    cudaFree(s->coef);
    cudaFree(s->p2);
    cudaFree(s->sc);
    s->work = s->coef = nullptr;
    s->p2 = nullptr;
    s->sc = nullptr;
    s->npw = std::max(npw, s->npw);
    s->nbnd = std::max(nbnd, s->nbnd);
    s->p2_ik = -1;
    bool ok = cudaMalloc((void**)&s->work, sizeof(double2) * 6 * (size_t)s->npw) == cudaSuccess &&
              cudaMalloc((void**)&s->coef, sizeof(double2) * (size_t)s->nbnd) == cudaSuccess &&
              cudaMalloc((void**)&s->p2, sizeof(double) * (size_t)s->npw) == cudaSuccess &&
              cudaMalloc((void**)&s->sc, sizeof(CgScalars)) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return fail(c, HPSI_ENOMEM, "cg_solve: workspace allocation failed");
    }
  }
  *out = s;
  return HPSI_OK;
}

// x -= Psi (Psi^H x) twice, Psi = the first i rows of psi (ld npw).
int orth_lower(Context& c, CgState& s, const double2* psi, int i, int npw, double2* x) {
  if (i == 0) return HPSI_OK;
  const cuDoubleComplex one = make_cuDoubleComplex(1.0, 0.0), zero = make_cuDoubleComplex(0.0, 0.0),
                        mone = make_cuDoubleComplex(-1.0, 0.0);
  auto Z = [](const double2* p) { return reinterpret_cast<const cuDoubleComplex*>(p); };
  for (int pass = 0; pass < 2; ++pass) {
    CBK(cublasZgemv(s.blas, CUBLAS_OP_C, npw, i, &one, Z(psi), npw, Z(x), 1, &zero,
                    reinterpret_cast<cuDoubleComplex*>(s.coef), 1),
        "zgemv projection");
    CBK(cublasZgemv(s.blas, CUBLAS_OP_N, npw, i, &mone, Z(psi), npw, Z(s.coef), 1, &one,
                    reinterpret_cast<cuDoubleComplex*>(x), 1),
        "zgemv projection update");
  }
  return HPSI_OK;
}

}  // namespace

int cg_run(Context& c, int ik, int nbnd, double tol, int maxiter, double2* psi, double* eig_out, int* iters_out,
           double* resnorm_out) {
  const Problem& p = c.probs[ik];
  const int npw = p.npw;
  CgState* s = nullptr;
  int rc = ensure_cg(c, npw, nbnd, &s);
  if (rc) return rc;
  double2* hpsi = s->work;
  double2* pg = hpsi + npw;
  double2* pg_prev = pg + npw;
  double2* ph = pg_prev + npw;
  double2* pn = ph + npw;
  double2* hpn = pn + npw;
  if (s->p2_ik != ik || s->p2_tmin != c.cg_tmin) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_cg_p2<<<(npw + 255) / 256, 256, 0, c.stream>>>(npw, p.d_kin, c.cg_tmin, s->p2)));
    s->p2_ik = ik;
    s->p2_tmin = c.cg_tmin;
  }
  long long steps_total = 0;
  bool all_converged = true;
  for (int i = 0; i < nbnd; ++i) {
    double2* x = psi + (size_t)i * npw;
    rc = orth_lower(c, *s, psi, i, npw, x);
    if (rc) return rc;
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_cg_normalize<<<1, kCgThreads, 0, c.stream>>>(npw, x, s->sc)));
    rc = apply_device(c, ik, x, hpsi, 1);
    if (rc) return rc;
    CgScalars h{};
    int steps = 0;
    for (;;) {
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_cg_state<<<1, kCgThreads, 0, c.stream>>>(npw, x, hpsi, s->p2, pg, s->sc)));
      CCK(cudaMemcpyAsync(&h, s->sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, c.stream), "cg_solve: scalar copy");
      CCK(cudaStreamSynchronize(c.stream), "cg_solve: step");
      rc = check_device_error(c);
      if (rc) return rc;
      if (!(h.n0 > 1e-28))
        return fail(c, HPSI_EINVAL, "cg_solve: the start vector of band " + std::to_string(i) +
                                        " lies in the span of the bands below it");
      if (!(std::sqrt(h.res2) > tol)) break;
      if (steps >= maxiter) {
        all_converged = false;
        break;
      }
      rc = orth_lower(c, *s, psi, i, npw, pg);
      if (rc) return rc;
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                  (k_cg_direction<<<1, kCgThreads, 0, c.stream>>>(npw, x, pg, pg_prev, ph, pn, s->sc)));
      rc = apply_device(c, ik, pn, hpn, 1);
      if (rc) return rc;
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_cg_move<<<1, kCgThreads, 0, c.stream>>>(npw, x, hpsi, pn, hpn, s->sc)));
      ++steps;
    }
    steps_total += steps;
    eig_out[i] = h.eps;
    if (resnorm_out) resnorm_out[i] = std::sqrt(h.res2);
  }
  if (iters_out) *iters_out = (int)std::min<long long>(steps_total, 0x7fffffff);
  if (!all_converged) return fail(c, HPSI_ENOTCONV, "cg_solve: a band reached maxiter");
  return HPSI_OK;
}

void cg_release(Context& c) {
  CgState* s = reinterpret_cast<CgState*>(c.cg);
  if (!s) return;
  cudaFree(s->work);
  cudaFree(s->coef);
  cudaFree(s->p2);
  cudaFree(s->sc);
  if (s->blas) cublasDestroy(s->blas);
  delete s;
  c.cg = nullptr;
}

}  // namespace hpsi
