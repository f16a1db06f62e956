// Block Davidson eigensolver around H|psi> (paper App. A.2.1), float64 on the GPU.
//
//   trial orbitals psi_i (orthonormal), eps_i = <psi_i|H|psi_i>
//   residuals      g_i = (H - eps_i) psi_i                      (S = I, norm-conserving)
//   corrections    delta psi_i = D g_i, <k+G|D|k+G'> = delta_GG' / (<k+G|H|k+G> - eps_i)
//   reduced basis  phi = {psi, delta psi, ...}, grown by the corrections of unconverged bands up
//                  to 4N vectors, then restarted from the N Ritz vectors
//   reduced problem sum_k (H_jk - eps S_jk) c_k = 0, psi_i <- sum_j c^(i)_j phi_j
//
// The basis is kept orthonormal: every block of corrections (each scaled to unit norm) is
// projected out of the basis twice (block Gram-Schmidt) and orthonormalised through the
// eigen-decomposition of its own overlap matrix, dropping directions whose overlap eigenvalue
// is below 1e-8.  A correction that loses all but 1e-3 of its norm to the projection lies in the
// basis up to rounding (this is what an exact diagonal D does: for a diagonal H, D g_i is
// parallel to psi_i); it is replaced by its raw residual g_i, which the Galerkin condition makes
// orthogonal to the basis.  S_jk is then the identity and the reduced problem is solved as a
// standard Hermitian one (cuSOLVER zheevd).
//
// The eps in D is eps_i per band by default (D approximates (H - eps_i S)^-1); option
// HPSI_OPT_PRECOND_SHIFT = 1 takes one eps for all bands, the highest Ritz value of the block
// (the "estimate of the highest occupied eigenvalue" of the diagonal form of D).  Subspace products are cuBLAS ZGEMMs (library GEMMs);
// residuals, norms and the preconditioner are the kernels below.  Only the residual norms and
// eigenvalues cross to the host each iteration.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "hpsi_internal.h"

namespace hpsi {

namespace {

constexpr double kDropAbs = 1e-8;     // overlap eigenvalues of unit corrections below this are dropped
constexpr double kCollapse = 1e-6;    // squared norm left after projection that marks a collapse

struct DavWork {
  int npw = 0, nbnd = 0, mmax = 0;
  double2* phi = nullptr;    // [mmax][npw]
  double2* hphi = nullptr;   // [mmax][npw]
  double2* psi = nullptr;    // [nbnd][npw] Ritz vectors
  double2* hpsi = nullptr;   // [nbnd][npw]
  double2* t = nullptr;      // [nbnd][npw] corrections / scratch
  double2* hsub = nullptr;   // [mmax][mmax] column-major
  double2* evec = nullptr;   // [mmax][mmax]
  double2* small = nullptr;  // [mmax][nbnd] coefficients
  double2* ovl = nullptr;    // [nbnd][nbnd] overlap scratch
  double* w = nullptr;       // [mmax] eigenvalues
  double* eps = nullptr;     // [nbnd]
  double* rnorm = nullptr;   // [nbnd]
  int* idx = nullptr;        // [nbnd] unconverged band list
  int* idx2 = nullptr;       // [nbnd] collapsed corrections
  double* cn2 = nullptr;     // [nbnd] squared norms of the corrections
  int* info = nullptr;
  double2* work = nullptr;
  int lwork = 0;
};

// R_i = HPsi_i - eps_i Psi_i (in place into R) and ||R_i||_2; one CTA per band.
__global__ void __launch_bounds__(256) k_residual(int npw, const double2* __restrict__ psi,
                                                  const double2* __restrict__ hpsi, const double* __restrict__ eps,
                                                  double2* __restrict__ r, double* __restrict__ rnorm) {
  const int b = blockIdx.x;
  const double e = eps[b];
  const double2* x = psi + (size_t)b * npw;
  const double2* hx = hpsi + (size_t)b * npw;
  double2* rb = r + (size_t)b * npw;
  double s = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double2 a = hx[g], v = x[g];
    const double2 q = make_double2(a.x - e * v.x, a.y - e * v.y);
    rb[g] = q;
    s += q.x * q.x + q.y * q.y;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) rnorm[b] = sqrt(red[0]);
}

// T_j = R_{idx[j]} / clamp(hdiag - eps_{idx[j]}), then T_j /= ||T_j||; one CTA per correction.
__global__ void __launch_bounds__(256) k_precondition(int npw, const int* __restrict__ idx,
                                                      const double2* __restrict__ r, const double* __restrict__ hdiag,
                                                      const double* __restrict__ eps, double tau, int eshift,
                                                      double2* __restrict__ t) {
  const int j = blockIdx.x;
  const int i = idx[j];
  const double e = eps[eshift >= 0 ? eshift : i];
  const double2* rb = r + (size_t)i * npw;
  double2* tb = t + (size_t)j * npw;
  double s = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    double x = hdiag[g] - e;
    if (fabs(x) < tau) x = x >= 0.0 ? tau : -tau;
    const double2 q = make_double2(rb[g].x / x, rb[g].y / x);
    tb[g] = q;
    s += q.x * q.x + q.y * q.y;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double nrm = red[0];
  const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) tb[g] = make_double2(tb[g].x * inv, tb[g].y * inv);
}

// ||t_j||^2 for each vector of a block; one CTA per vector.
__global__ void __launch_bounds__(256) k_norm2(int npw, const double2* __restrict__ t, double* __restrict__ out) {
  const double2* tb = t + (size_t)blockIdx.x * npw;
  double s = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) s += tb[g].x * tb[g].x + tb[g].y * tb[g].y;
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// t_j <- r_{idx[j]} / ||r_{idx[j]}|| for the listed j (collapsed corrections); one CTA per entry.
__global__ void k_fallback(int npw, const int* __restrict__ which, const int* __restrict__ idx,
                           const double2* __restrict__ r, const double* __restrict__ rnorm, double2* __restrict__ t) {
  const int j = which[blockIdx.x];
  const int i = idx[j];
  const double s = 1.0 / rnorm[i];
  const double2* rb = r + (size_t)i * npw;
  double2* tb = t + (size_t)j * npw;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) tb[g] = make_double2(rb[g].x * s, rb[g].y * s);
}

// Columns of the eigenvector matrix V (n x n, ld) scaled by 1/sqrt(lambda) for kept directions,
// compacted into out[n][nkeep] (column-major, ld n): out[:, c] = V[:, first + c] / sqrt(w[first + c]).
__global__ void k_canon_scale(int n, int ld, int first, int nkeep, const double2* __restrict__ v,
                              const double* __restrict__ w, double2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nkeep) return;
  const int row = i % n, c = i / n;
  const double s = 1.0 / sqrt(w[first + c]);
  const double2 x = v[(size_t)(first + c) * ld + row];
  out[(size_t)c * n + row] = make_double2(x.x * s, x.y * s);
}

__global__ void k_copy_matrix(int rows, int cols, const double2* __restrict__ src, int lds, double2* __restrict__ dst,
                              int ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i % rows, c = i / rows;
  dst[(size_t)c * ldd + r] = src[(size_t)c * lds + r];
}

const cuDoubleComplex kOne = {1.0, 0.0};
const cuDoubleComplex kZero = {0.0, 0.0};
const cuDoubleComplex kMinusOne = {-1.0, 0.0};

inline cuDoubleComplex* Z(double2* p) { return reinterpret_cast<cuDoubleComplex*>(p); }
inline const cuDoubleComplex* Z(const double2* p) { return reinterpret_cast<const cuDoubleComplex*>(p); }

}  // namespace

struct DavHandles {
  cublasHandle_t blas = nullptr;
  cusolverDnHandle_t solver = nullptr;
  DavWork wk;
};

static int blas_fail(Context& c, int st, const char* what) {
  c.err = std::string(what) + " failed with status " + std::to_string(st);
  return HPSI_ECUDA;
}

#define DCK(x, what)                                            \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what);       \
  } while (0)
#define BCK(x, what)                                            \
  do {                                                          \
    int s_ = (int)(x);                                          \
    if (s_ != 0) return blas_fail(c, s_, what);                 \
  } while (0)

static void free_work(DavWork& w) {
  cudaFree(w.phi);
  cudaFree(w.hphi);
  cudaFree(w.psi);
  cudaFree(w.hpsi);
  cudaFree(w.t);
  cudaFree(w.hsub);
  cudaFree(w.evec);
  cudaFree(w.small);
  cudaFree(w.ovl);
  cudaFree(w.w);
  cudaFree(w.eps);
  cudaFree(w.rnorm);
  cudaFree(w.idx);
  cudaFree(w.idx2);
  cudaFree(w.cn2);
  cudaFree(w.info);
  cudaFree(w.work);
  w = DavWork();
}

void davidson_release(Context& c) {
  DavHandles* h = reinterpret_cast<DavHandles*>(c.blas);
  if (!h) return;
  free_work(h->wk);
  if (h->blas) cublasDestroy(h->blas);
  if (h->solver) cusolverDnDestroy(h->solver);
  delete h;
  c.blas = nullptr;
}

static int alloc_work(Context& c, DavHandles& h, int npw, int nbnd) {
  DavWork& w = h.wk;
  const int mmax = 4 * nbnd;
  if (w.npw == npw && w.nbnd == nbnd) return HPSI_OK;
  free_work(w);
  w.npw = npw;
  w.nbnd = nbnd;
  w.mmax = mmax;
  auto al = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  const size_t v = sizeof(double2) * (size_t)npw;
  bool ok = al((void**)&w.phi, v * mmax) && al((void**)&w.hphi, v * mmax) && al((void**)&w.psi, v * nbnd) &&
            al((void**)&w.hpsi, v * nbnd) && al((void**)&w.t, v * nbnd) &&
            al((void**)&w.hsub, sizeof(double2) * (size_t)mmax * mmax) &&
            al((void**)&w.evec, sizeof(double2) * (size_t)mmax * mmax) &&
            al((void**)&w.small, sizeof(double2) * (size_t)mmax * nbnd) &&
            al((void**)&w.ovl, sizeof(double2) * (size_t)nbnd * nbnd) && al((void**)&w.w, sizeof(double) * mmax) &&
            al((void**)&w.eps, sizeof(double) * nbnd) && al((void**)&w.rnorm, sizeof(double) * nbnd) &&
            al((void**)&w.idx, sizeof(int) * nbnd) && al((void**)&w.idx2, sizeof(int) * nbnd) &&
            al((void**)&w.cn2, sizeof(double) * nbnd) && al((void**)&w.info, sizeof(int));
  if (!ok) {
    free_work(w);
    return fail(c, HPSI_ENOMEM, "davidson_solve: device allocation of the reduced basis failed");
  }
  int lw = 0;
  BCK(cusolverDnZheevd_bufferSize(h.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, mmax, Z(w.evec), mmax,
                                  w.w, &lw),
      "cusolverDnZheevd_bufferSize");
  w.lwork = lw;
  if (!al((void**)&w.work, sizeof(double2) * (size_t)std::max(lw, 1))) {
    free_work(w);
    return fail(c, HPSI_ENOMEM, "davidson_solve: workspace allocation failed");
  }
  return HPSI_OK;
}

// eigen-decomposition of the leading n x n block of a (ld) into w.evec / w.w (ascending)
static int small_eigh(Context& c, DavHandles& h, const double2* a, int lda, int n) {
  DavWork& w = h.wk;
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_copy_matrix<<<(n * n + 255) / 256, 256, 0, c.stream>>>(n, n, a, lda, w.evec, n)));
  BCK(cusolverDnZheevd(h.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, Z(w.evec), n, w.w, Z(w.work),
                       w.lwork, w.info),
      "cusolverDnZheevd");
  int info = 0;
  DCK(cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "davidson info copy");
  DCK(cudaStreamSynchronize(c.stream), "davidson eigensolve");
  if (info != 0) return fail(c, HPSI_ESINGULAR, "zheevd of the reduced matrix failed, info " + std::to_string(info));
  return HPSI_OK;
}

// Orthonormalise the block x[0:n] (band-major, npw) against itself: overlap S = x^H x, S = V L V^H,
// x <- x V_keep L_keep^{-1/2}, keeping directions with L > thr (thr relative to max(L) when
// relative is set).  The result (nkeep vectors) goes to out, which must not overlap x.
static int canonical_orth(Context& c, DavHandles& h, const double2* x, int n, double2* out, int* nkeep, double thr,
                          bool relative) {
  DavWork& w = h.wk;
  const int npw = w.npw;
  BCK(cublasZgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, n, n, npw, &kOne, Z(x), npw, Z(x), npw, &kZero, Z(w.ovl), n),
      "zgemm overlap");
  // evec / w receive the decomposition of the overlap (the Ritz vectors were formed already)
  int rc = small_eigh(c, h, w.ovl, n, n);
  if (rc) return rc;
  std::vector<double> lam(n);
  DCK(cudaMemcpyAsync(lam.data(), w.w, sizeof(double) * n, cudaMemcpyDeviceToHost, c.stream), "overlap eigenvalues");
  DCK(cudaStreamSynchronize(c.stream), "overlap eigenvalues");
  const double cut = relative ? thr * lam[n - 1] : thr;
  int first = 0;
  while (first < n && !(lam[first] > cut && lam[first] > 1e-300)) ++first;
  const int nk = n - first;
  *nkeep = nk;
  if (nk == 0) return HPSI_OK;
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_canon_scale<<<(n * nk + 255) / 256, 256, 0, c.stream>>>(n, n, first, nk, w.evec, w.w, w.small)));
  BCK(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nk, n, &kOne, Z(x), npw, Z(w.small), n, &kZero, Z(out), npw),
      "zgemm orthonormalise");
  return HPSI_OK;
}

int davidson_run(Context& c, int ik, int nbnd, double tol, int maxiter, double2* psio, double* eig_out, int* iters_out,
                 double* resnorm_out) {
  const Problem& p = c.probs[ik];
  DavHandles* h = reinterpret_cast<DavHandles*>(c.blas);
  if (!h) {
    h = new DavHandles();
    c.blas = h;
    BCK(cublasCreate(&h->blas), "cublasCreate");
    BCK(cusolverDnCreate(&h->solver), "cusolverDnCreate");
  }
  BCK(cublasSetStream(h->blas, c.stream), "cublasSetStream");
  BCK(cusolverDnSetStream(h->solver, c.stream), "cusolverDnSetStream");
  int rc = alloc_work(c, *h, p.npw, nbnd);
  if (rc) return rc;
  DavWork& w = h->wk;
  const int npw = p.npw, N = nbnd, mmax = w.mmax;
  const size_t vb = sizeof(double2) * (size_t)npw;

  // phi[0:N] <- orthonormalised initial guess
  int nk = 0;
  rc = canonical_orth(c, *h, psio, N, w.phi, &nk, 1e-12, true);
  if (rc) return rc;
  if (nk < N) return fail(c, HPSI_EINVAL, "davidson_solve: initial guess is linearly dependent");
  rc = apply_device(c, ik, w.phi, w.hphi, N);
  if (rc) return rc;
  int m = N;
  BCK(cublasZgemm(h->blas, CUBLAS_OP_C, CUBLAS_OP_N, m, m, npw, &kOne, Z(w.phi), npw, Z(w.hphi), npw, &kZero,
                  Z(w.hsub), mmax),
      "zgemm H_sub");
  std::vector<double> rn(N), ev(N);
  std::vector<int> uidx(N);
  int it = 0;
  bool converged = false;
  for (;;) {
    rc = small_eigh(c, *h, w.hsub, mmax, m);
    if (rc) return rc;
    // Ritz vectors psi = phi C[:, 0:N], hpsi = hphi C[:, 0:N]
    BCK(cublasZgemm(h->blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, N, m, &kOne, Z(w.phi), npw, Z(w.evec), m, &kZero,
                    Z(w.psi), npw),
        "zgemm Ritz vectors");
    BCK(cublasZgemm(h->blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, N, m, &kOne, Z(w.hphi), npw, Z(w.evec), m, &kZero,
                    Z(w.hpsi), npw),
        "zgemm H Ritz vectors");
    DCK(cudaMemcpyAsync(w.eps, w.w, sizeof(double) * N, cudaMemcpyDeviceToDevice, c.stream), "eps copy");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_residual<<<N, 256, 0, c.stream>>>(npw, w.psi, w.hpsi, w.eps, w.t, w.rnorm)));
    DCK(cudaGetLastError(), "residual kernel");
    DCK(cudaMemcpyAsync(rn.data(), w.rnorm, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream), "norm copy");
    DCK(cudaMemcpyAsync(ev.data(), w.eps, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream), "eig copy");
    DCK(cudaStreamSynchronize(c.stream), "davidson iteration");
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
    if (m + nc > mmax) {
      // restart from the Ritz vectors
      DCK(cudaMemcpyAsync(w.phi, w.psi, vb * N, cudaMemcpyDeviceToDevice, c.stream), "restart copy");
      DCK(cudaMemcpyAsync(w.hphi, w.hpsi, vb * N, cudaMemcpyDeviceToDevice, c.stream), "restart copy");
      m = N;
      BCK(cublasZgemm(h->blas, CUBLAS_OP_C, CUBLAS_OP_N, m, m, npw, &kOne, Z(w.phi), npw, Z(w.hphi), npw, &kZero,
                      Z(w.hsub), mmax),
          "zgemm H_sub restart");
    }
    DCK(cudaMemcpyAsync(w.idx, uidx.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, c.stream), "index copy");
    // corrections into phi[m : m+nc] (t holds the residuals)
    double2* tnew = w.phi + (size_t)m * npw;
    const int eshift = c.opt_shift == 1 ? N - 1 : -1;
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_precondition<<<nc, 256, 0, c.stream>>>(npw, w.idx, w.t, p.d_hdiag, w.eps, c.opt_tau, eshift, tnew)));
    DCK(cudaGetLastError(), "precondition kernel");
    for (int round = 0; round < 2; ++round) {
      // two passes of block Gram-Schmidt against phi[0:m]
      for (int pass = 0; pass < 2; ++pass) {
        BCK(cublasZgemm(h->blas, CUBLAS_OP_C, CUBLAS_OP_N, m, nc, npw, &kOne, Z(w.phi), npw, Z(tnew), npw, &kZero,
                        Z(w.small), m),
            "zgemm projection");
        BCK(cublasZgemm(h->blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nc, m, &kMinusOne, Z(w.phi), npw, Z(w.small), m,
                        &kOne, Z(tnew), npw),
            "zgemm projection update");
      }
      if (round == 1) break;
      // corrections that lie in the basis are replaced by their raw residuals
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_norm2<<<nc, 256, 0, c.stream>>>(npw, tnew, w.cn2)));
      std::vector<double> cn(nc);
      DCK(cudaMemcpyAsync(cn.data(), w.cn2, sizeof(double) * nc, cudaMemcpyDeviceToHost, c.stream), "norm copy");
      DCK(cudaStreamSynchronize(c.stream), "correction norms");
      std::vector<int> col;
      for (int j = 0; j < nc; ++j)
        if (!(cn[j] >= kCollapse)) col.push_back(j);
      if (col.empty()) break;
      DCK(cudaMemcpyAsync(w.idx2, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice, c.stream),
          "index copy");
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_fallback<<<(int)col.size(), 256, 0, c.stream>>>(npw, w.idx2, w.idx, w.t, w.rnorm, tnew)));
      DCK(cudaGetLastError(), "fallback kernel");
    }
    // orthonormalise the block itself (w.t is free now: residuals were consumed)
    int nkeep = 0;
    rc = canonical_orth(c, *h, tnew, nc, w.t, &nkeep, kDropAbs, false);
    if (rc) return rc;
    if (nkeep == 0) {
      // nothing new can be added: the residuals lie in the basis up to rounding
      converged = rmax <= tol;
      break;
    }
    DCK(cudaMemcpyAsync(tnew, w.t, vb * nkeep, cudaMemcpyDeviceToDevice, c.stream), "basis copy");
    rc = apply_device(c, ik, tnew, w.hphi + (size_t)m * npw, nkeep);
    if (rc) return rc;
    // new columns of H_sub: phi[0:m+nkeep]^H hphi[m:m+nkeep]  (upper triangle is what zheevd reads)
    BCK(cublasZgemm(h->blas, CUBLAS_OP_C, CUBLAS_OP_N, m + nkeep, nkeep, npw, &kOne, Z(w.phi), npw,
                    Z(w.hphi + (size_t)m * npw), npw, &kZero, Z(w.hsub + (size_t)m * mmax), mmax),
        "zgemm H_sub columns");
    m += nkeep;
  }
  DCK(cudaMemcpyAsync(psio, w.psi, vb * N, cudaMemcpyDeviceToDevice, c.stream), "eigenvector copy");
  DCK(cudaStreamSynchronize(c.stream), "davidson end");
  for (int i = 0; i < N; ++i) eig_out[i] = ev[i];
  if (resnorm_out)
    for (int i = 0; i < N; ++i) resnorm_out[i] = rn[i];
  if (iters_out) *iters_out = it;
  if (!converged) return fail(c, HPSI_ENOTCONV, "davidson_solve: not converged within maxiter");
  return HPSI_OK;
}

}  // namespace hpsi
