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
// projected out of the basis twice (block Gram-Schmidt) and orthonormalised by Cholesky QR of its
// own overlap (float64 factor) when every squared pivot exceeds 1e-6, otherwise through the
// eigen-decomposition of the overlap, dropping directions whose overlap eigenvalue is below 1e-8.  A correction that loses all but 1e-3 of its norm to the projection lies in the
// basis up to rounding (this is what an exact diagonal D does: for a diagonal H, D g_i is
// parallel to psi_i); it is replaced by its raw residual g_i, which the Galerkin condition makes
// orthogonal to the basis.  S_jk is then the identity and the reduced problem is solved as a
// standard Hermitian one (cuSOLVER zheevd).
//
// Mixed precision (HPSI_MIXED): the reduced basis and its products are complex64 (cuBLAS CGEMM);
// the small eigenproblems, the residual norms and the final eigenvalues are float64 -- at exit H
// is applied once more to the Ritz vectors, with the float64 operator unless HPSI_OPT_FINAL_FP64
// is 0, and eps_i = <psi_i|H psi_i> / <psi_i|psi_i> is summed in float64: the eigenvalue error
// is then second order in the eigenvector error left by the mixed iterations.
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
constexpr double kReorth = 0.5;       // squared norm a unit correction keeps after one projection pass
                                      // below which a second pass runs (Daniel-Gragg-Kaufman-Stewart)
constexpr int kStall = 8;             // mixed thick restart: iterations without progress before plain restarts

struct DavWork {
  int npw = 0, nbnd = 0, mmax = 0;
  double2* phi = nullptr;    // [mmax][npw]
  double2* hphi = nullptr;   // [mmax][npw]
  double2* psi = nullptr;    // [nbnd][npw] Ritz vectors
  double2* hpsi = nullptr;   // [nbnd][npw]
  double2* t = nullptr;      // [nbnd][npw] corrections / scratch
  double2* rst = nullptr;    // [kmax][npw] restart scratch
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
  // mixed path: float32 basis and products, float64 staging for H|psi>
  bool mixed = false;
  float2* phi32 = nullptr;    // [mmax][npw]
  float2* hphi32 = nullptr;   // [mmax][npw]
  float2* psi32 = nullptr;    // [nbnd][npw]
  float2* hpsi32 = nullptr;   // [nbnd][npw]
  float2* t32 = nullptr;      // [nbnd][npw]
  float2* lock32 = nullptr;   // [nbnd][npw] hard-locked Ritz vectors
  int kmax = 0;               // most Ritz vectors a restart keeps: max(nbnd, mmax / 2)
  float2* ysub32 = nullptr;   // [kmax][mmax] reduced eigenvectors of the kept Ritz vectors
  float2* rst32 = nullptr;    // [kmax][npw] restart scratch
  int* sel = nullptr;         // [kmax] Ritz indices a restart keeps
  float2* part32 = nullptr;   // K-chunk partial products of the Ritz and restart GEMMs
  size_t part_cap = 0;        // elements of part32
  float2* small32 = nullptr;  // [mmax][nbnd]
  float2* ovl32 = nullptr;    // [nbnd][nbnd]
  float2* hcol32 = nullptr;   // [kmax][mmax] H_sub columns in float32
  float* hdiag32 = nullptr;   // [npw] float copy of <k+G|H|k+G>
  SplitBasis phi_split, hphi_split;   // bf16 splits of the basis for the tensor-core products
  SubspaceGemm sg;
  TcInner tci;                // tcgen05 inner products (HPSI_OPT_FP32_GEMM = 4); caches phi32's split
  double2* in64 = nullptr;    // [nbnd][npw]
  double2* out64 = nullptr;   // [nbnd][npw]
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
    const double inv = 1.0 / x;
    const double2 q = make_double2(rb[g].x * inv, rb[g].y * inv);
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
  cudaFree(w.rst);
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
  cudaFree(w.phi32);
  cudaFree(w.hphi32);
  cudaFree(w.psi32);
  cudaFree(w.hpsi32);
  cudaFree(w.t32);
  cudaFree(w.lock32);
  cudaFree(w.ysub32);
  cudaFree(w.rst32);
  cudaFree(w.sel);
  cudaFree(w.part32);
  cudaFree(w.small32);
  cudaFree(w.ovl32);
  cudaFree(w.hcol32);
  cudaFree(w.hdiag32);
  w.phi_split.release();
  w.hphi_split.release();
  w.sg.release();
  w.tci.release();
  cudaFree(w.in64);
  cudaFree(w.out64);
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

static int alloc_work(Context& c, DavHandles& h, int npw, int nbnd, bool mixed) {
  DavWork& w = h.wk;
  const int mmax = basis_of(c) * nbnd;
  if (w.npw == npw && w.nbnd == nbnd && w.mixed == mixed && w.mmax == mmax) return HPSI_OK;
  free_work(w);
  w.npw = npw;
  w.nbnd = nbnd;
  w.mmax = mmax;
  w.mixed = mixed;
  auto al = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  const size_t v = sizeof(double2) * (size_t)npw;
  const size_t v32 = sizeof(float2) * (size_t)npw;
  w.kmax = std::max(nbnd, mmax / 2);
  bool ok = al((void**)&w.hsub, sizeof(double2) * (size_t)mmax * mmax) &&
            al((void**)&w.evec, sizeof(double2) * (size_t)mmax * mmax) &&
            al((void**)&w.small, sizeof(double2) * (size_t)mmax * nbnd) &&
            al((void**)&w.ovl, sizeof(double2) * (size_t)nbnd * nbnd) && al((void**)&w.w, sizeof(double) * mmax) &&
            al((void**)&w.eps, sizeof(double) * nbnd) && al((void**)&w.rnorm, sizeof(double) * nbnd) &&
            al((void**)&w.idx, sizeof(int) * nbnd) && al((void**)&w.idx2, sizeof(int) * nbnd) &&
            al((void**)&w.cn2, sizeof(double) * nbnd) && al((void**)&w.info, sizeof(int));
  if (ok && !mixed)
    ok = al((void**)&w.phi, v * mmax) && al((void**)&w.hphi, v * mmax) && al((void**)&w.psi, v * nbnd) &&
         al((void**)&w.hpsi, v * nbnd) && al((void**)&w.t, v * nbnd) && al((void**)&w.rst, v * w.kmax);
  if (ok && mixed)
    ok = al((void**)&w.ysub32, sizeof(float2) * (size_t)mmax * w.kmax) && al((void**)&w.rst32, v32 * w.kmax) &&
         al((void**)&w.sel, sizeof(int) * w.kmax) &&
         al((void**)&w.phi32, v32 * mmax) && al((void**)&w.hphi32, v32 * mmax) && al((void**)&w.psi32, v32 * nbnd) &&
         al((void**)&w.hpsi32, v32 * nbnd) && al((void**)&w.t32, v32 * nbnd) && al((void**)&w.lock32, v32 * nbnd) &&
         al((void**)&w.small32, sizeof(float2) * (size_t)mmax * nbnd) &&
         al((void**)&w.ovl32, sizeof(float2) * (size_t)nbnd * nbnd) &&
         al((void**)&w.hcol32, sizeof(float2) * (size_t)mmax * w.kmax) && al((void**)&w.hdiag32, sizeof(float) * npw) && al((void**)&w.in64, v * nbnd) &&
         al((void**)&w.out64, v * nbnd);
  if (!ok) {
    free_work(w);
    return fail(c, HPSI_ENOMEM, "davidson_solve: device allocation of the reduced basis failed");
  }
  int lw = 0, lw2 = 0, lw3 = 0, meig = 0;
  BCK(cusolverDnZheevd_bufferSize(h.solver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, mmax, Z(w.evec), mmax,
                                  w.w, &lw),
      "cusolverDnZheevd_bufferSize");
  BCK(cusolverDnZheevdx_bufferSize(h.solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_UPPER,
                                   mmax, Z(w.evec), mmax, 0.0, 0.0, 1, nbnd, &meig, w.w, &lw2),
      "cusolverDnZheevdx_bufferSize");
  BCK(cusolverDnZpotrf_bufferSize(h.solver, CUBLAS_FILL_MODE_UPPER, nbnd, Z(w.ovl), nbnd, &lw3),
      "cusolverDnZpotrf_bufferSize");
  w.lwork = std::max(lw, std::max(lw2, lw3));
  lw = w.lwork;
  if (!al((void**)&w.work, sizeof(double2) * (size_t)std::max(lw, 1))) {
    free_work(w);
    return fail(c, HPSI_ENOMEM, "davidson_solve: workspace allocation failed");
  }
  return HPSI_OK;
}

// eigen-decomposition of the leading n x n block of a (ld) into w.evec / w.w (ascending)
static int small_eigh(Context& c, DavHandles& h, const double2* a, int lda, int n) {
  DavWork& w = h.wk;
  return eigh_reduced(c, a, lda, n, n, w.w, w.evec);
}

// Lowest nwant eigenpairs of the leading n x n block of a (ld): values in w.w, vectors in the first
// nwant columns of w.evec (ld n).
static int lowest_eigh(Context& c, DavHandles& h, const double2* a, int lda, int n, int nwant) {
  DavWork& w = h.wk;
  if (c.eigensolver == 1) {
    bool fallback = false;
    const int rc = eigh_lowest(c, a, lda, n, nwant, w.w, w.evec, &fallback);
    if (rc || !fallback) return rc;
  }
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_copy_matrix<<<(n * n + 255) / 256, 256, 0, c.stream>>>(n, n, a, lda, w.evec, n)));
  int meig = 0;
  BCK(cusolverDnZheevdx(h.solver, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_UPPER, n,
                        Z(w.evec), n, 0.0, 0.0, 1, nwant, &meig, w.w, Z(w.work), w.lwork, w.info),
      "cusolverDnZheevdx");
  int info = 0;
  DCK(cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "davidson info copy");
  DCK(cudaStreamSynchronize(c.stream), "davidson eigensolve");
  if (info != 0 || meig < nwant)
    return fail(c, HPSI_ESINGULAR, "zheevdx of the reduced matrix failed, info " + std::to_string(info));
  return HPSI_OK;
}

// |U_ii|^2 of an n x n upper factor (ld n) into out[n]
__global__ void k_diag2(int n, const double2* __restrict__ u, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = u[(size_t)i * n + i].x * u[(size_t)i * n + i].x + u[(size_t)i * n + i].y * u[(size_t)i * n + i].y;
}

// Cholesky of the float64 overlap in w.ovl (n x n, ld n): true if it succeeded with every |U_ii|^2
// above thr (relative to the largest when relative), i.e. the block is safely independent.
static int chol_overlap(Context& c, DavHandles& h, int n, double thr, bool relative, bool* ok) {
  DavWork& w = h.wk;
  *ok = false;
  BCK(cusolverDnZpotrf(h.solver, CUBLAS_FILL_MODE_UPPER, n, Z(w.ovl), n, Z(w.work), w.lwork, w.info),
      "cusolverDnZpotrf");
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_diag2<<<(n + 255) / 256, 256, 0, c.stream>>>(n, w.ovl, w.cn2)));
  int info = 0;
  std::vector<double> dg(n);
  DCK(cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, c.stream), "potrf info copy");
  DCK(cudaMemcpyAsync(dg.data(), w.cn2, sizeof(double) * n, cudaMemcpyDeviceToHost, c.stream), "potrf diag copy");
  DCK(cudaStreamSynchronize(c.stream), "potrf");
  if (info != 0) return HPSI_OK;
  double mx = 0.0, mn = 1e300;
  for (double v : dg) {
    mx = std::max(mx, v);
    mn = std::min(mn, v);
  }
  *ok = mn > (relative ? thr * mx : thr);
  return HPSI_OK;
}

// Orthonormalise the block x[0:n] (band-major, npw) against itself: overlap S = x^H x, S = V L V^H,
// x <- x V_keep L_keep^{-1/2}, keeping directions with L > thr (thr relative to max(L) when
// relative is set).  The result (nkeep vectors) goes to out, which must not overlap x.
static int canonical_orth(Context& c, DavHandles& h, const double2* x, int n, double2* out, int* nkeep, double thr,
                          bool relative) {
  DavWork& w = h.wk;
  const int npw = w.npw;
  // Cholesky QR when the block is well conditioned: x <- x U^-1 with S = U^H U
  BCK(cublasZgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, n, n, npw, &kOne, Z(x), npw, Z(x), npw, &kZero, Z(w.ovl), n),
      "zgemm overlap");
  bool chol_ok = false;
  int rc0 = chol_overlap(c, h, n, relative ? 1e-10 : 1e-6, relative, &chol_ok);
  if (rc0) return rc0;
  if (chol_ok) {
    DCK(cudaMemcpyAsync(out, x, sizeof(double2) * (size_t)n * npw, cudaMemcpyDeviceToDevice, c.stream), "copy");
    BCK(cublasZtrsm(h.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, npw, n,
                    &kOne, Z(w.ovl), n, Z(out), npw),
        "ztrsm");
    *nkeep = n;
    return HPSI_OK;
  }
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

// ---- mixed path: float32 basis, float64 small problems, norms and Rayleigh quotients ----------

namespace {

// Sum over a block of up to 1024 threads: warp shuffles, then warp 0 reduces the per-warp values
// (one float64 chain of depth 10 instead of every thread adding all partials); red holds >= 33.
__device__ __forceinline__ double block_sum256(double s, double* red) {
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

// Neumaier's compensated summation in float32: the running error of each addition is kept in c,
// so a thread's partial sum of positive float32 terms is accurate to about one float32 rounding
// of the total, whatever the number of terms.
struct CompSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += fabsf(s) >= fabsf(x) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Sum of squares of float32 values to float64 accuracy without a float64 instruction per element:
// each square split exactly by an FMA (q^2 = p + e) and accumulated in a (hi, lo) pair of floats
// through TwoSum; the _rn intrinsics keep the compiler from contracting or reassociating it.
struct SqSum {
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

// R_i = HPsi_i - eps_i Psi_i (float32 data) and ||R_i||_2 to float64 accuracy (SqSum partial sums,
// float64 across threads); one CTA per band.  eps = e_hi + e_lo in two floats keeps hpsi - eps psi
// at float32 accuracy of the (small) result.
__global__ void __launch_bounds__(1024) k_residual32(int npw, const float2* __restrict__ psi,
                                                    const float2* __restrict__ hpsi, const double* __restrict__ eps,
                                                    float2* __restrict__ r, double* __restrict__ rnorm) {
  __shared__ double red[33];
  const int b = blockIdx.x;
  const double e = eps[b];
  const float ehi = (float)e, elo = (float)(e - (double)ehi);
  const float2* x = psi + (size_t)b * npw;
  const float2* hx = hpsi + (size_t)b * npw;
  float2* rb = r + (size_t)b * npw;
  SqSum cs;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const float2 xv = x[g], hv = hx[g];
    const float qx = fmaf(-elo, xv.x, fmaf(-ehi, xv.x, hv.x));
    const float qy = fmaf(-elo, xv.y, fmaf(-ehi, xv.y, hv.y));
    rb[g] = make_float2(qx, qy);
    cs.add(qx);
    cs.add(qy);
  }
  const double s = block_sum256(cs.value(), red);
  if (threadIdx.x == 0) rnorm[b] = sqrt(s);
}

// T_j = R_{idx[j]} / clamp(hdiag - eps), then T_j /= ||T_j||, in float32 (hdiag32 is the float copy
// of the diagonal of H); one CTA per correction.
__global__ void __launch_bounds__(1024) k_precondition32(int npw, const int* __restrict__ idx,
                                                        const float2* __restrict__ r, const float* __restrict__ hdiag32,
                                                        const double* __restrict__ eps, double tau, int eshift,
                                                        float2* __restrict__ t) {
  __shared__ double red[33];
  const int j = blockIdx.x;
  const int i = idx[j];
  const float e = (float)eps[eshift >= 0 ? eshift : i];
  const float tf = (float)tau;
  const float2* rb = r + (size_t)i * npw;
  float2* tb = t + (size_t)j * npw;
  CompSum cs;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    float x = hdiag32[g] - e;
    if (fabsf(x) < tf) x = x >= 0.f ? tf : -tf;
    const float inv = 1.0f / x;
    const float2 rv = rb[g];
    const float qx = rv.x * inv, qy = rv.y * inv;
    tb[g] = make_float2(qx, qy);
    cs.add(fmaf(qx, qx, qy * qy));
  }
  const double s = block_sum256(cs.value(), red);
  const float inv = s > 0.0 ? (float)(1.0 / sqrt(s)) : 0.f;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) tb[g] = make_float2(tb[g].x * inv, tb[g].y * inv);
}

__global__ void __launch_bounds__(1024) k_norm2_32(int npw, const float2* __restrict__ t, double* __restrict__ out) {
  __shared__ double red[33];
  const float2* tb = t + (size_t)blockIdx.x * npw;
  SqSum cs;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const float2 v = tb[g];
    cs.add(v.x);
    cs.add(v.y);
  }
  const double s = block_sum256(cs.value(), red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

__global__ void k_fallback32(int npw, const int* __restrict__ which, const int* __restrict__ idx,
                             const float2* __restrict__ r, const double* __restrict__ rnorm, float2* __restrict__ t) {
  const int j = which[blockIdx.x];
  const int i = idx[j];
  const float s = (float)(1.0 / rnorm[i]);
  const float2* rb = r + (size_t)i * npw;
  float2* tb = t + (size_t)j * npw;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) tb[g] = make_float2(rb[g].x * s, rb[g].y * s);
}

__global__ void k_canon_scale32(int n, int ld, int first, int nkeep, const double2* __restrict__ v,
                                const double* __restrict__ w, float2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * nkeep) return;
  const int row = i % n, c = i / n;
  const double s = 1.0 / sqrt(w[first + c]);
  const double2 x = v[(size_t)(first + c) * ld + row];
  out[(size_t)c * n + row] = make_float2((float)(x.x * s), (float)(x.y * s));
}

__global__ void k_cvt_64_32(size_t n, const double2* __restrict__ in, float2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

__global__ void k_cvt_d2f(int n, const double* __restrict__ in, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

__global__ void k_cvt_32_64(size_t n, const float2* __restrict__ in, double2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

__global__ void k_mat_32_to_64(int rows, int cols, const float2* __restrict__ src, int lds, double2* __restrict__ dst,
                               int ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i % rows, c = i / rows;
  const float2 x = src[(size_t)c * lds + r];
  dst[(size_t)c * ldd + r] = make_double2((double)x.x, (double)x.y);
}

__global__ void k_mat_64_to_32(int rows, int cols, const double2* __restrict__ src, int lds, float2* __restrict__ dst,
                               int ldd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const int r = i % rows, c = i / rows;
  const double2 x = src[(size_t)c * lds + r];
  dst[(size_t)c * ldd + r] = make_float2((float)x.x, (float)x.y);
}

// eps_i = Re<psi_i|H psi_i> / <psi_i|psi_i> and ||H psi_i - eps_i psi_i|| / ||psi_i||, float64.
__global__ void __launch_bounds__(1024) k_rayleigh(int npw, const double2* __restrict__ psi,
                                                  const double2* __restrict__ hpsi, double* __restrict__ eps,
                                                  double* __restrict__ rnorm) {
  __shared__ double red[33];
  const int b = blockIdx.x;
  const double2* x = psi + (size_t)b * npw;
  const double2* hx = hpsi + (size_t)b * npw;
  double xx = 0.0, xh = 0.0, hh = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    xx += x[g].x * x[g].x + x[g].y * x[g].y;
    xh += x[g].x * hx[g].x + x[g].y * hx[g].y;
    hh += hx[g].x * hx[g].x + hx[g].y * hx[g].y;
  }
  xx = block_sum256(xx, red);
  xh = block_sum256(xh, red);
  hh = block_sum256(hh, red);
  if (threadIdx.x == 0) {
    const double e = xh / xx;
    eps[b] = e;
    // ||Hx - e x||^2 = hh - 2 e xh + e^2 xx, evaluated directly below for accuracy
  }
  __syncthreads();
  const double e = xh / xx;
  double rr = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) {
    const double qx = hx[g].x - e * x[g].x, qy = hx[g].y - e * x[g].y;
    rr += qx * qx + qy * qy;
  }
  rr = block_sum256(rr, red);
  if (threadIdx.x == 0) rnorm[b] = sqrt(rr / xx);
}

__global__ void k_gather_rows(int npw, const int* __restrict__ perm, const double2* __restrict__ src,
                              double2* __restrict__ dst) {
  const int b = blockIdx.x;
  const double2* s = src + (size_t)perm[b] * npw;
  double2* o = dst + (size_t)b * npw;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) o[g] = s[g];
}

// dst[b] = src[sel[b]] and, if given, dst2[b] = src2[sel[b]]; one CTA per row, rows of npw.
__global__ void k_gather_rows32(int npw, const int* __restrict__ sel, const float2* __restrict__ src,
                                float2* __restrict__ dst, const float2* __restrict__ src2, float2* __restrict__ dst2) {
  const int b = blockIdx.x;
  const size_t from = (size_t)sel[b] * npw, to = (size_t)b * npw;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) dst[to + g] = src[from + g];
  if (src2)
    for (int g = threadIdx.x; g < npw; g += blockDim.x) dst2[to + g] = src2[from + g];
}

// y[:, j] = float(v[:, sel[j]]) for the rows 0..rows-1 (column-major, ld rows for both).
__global__ void k_select_columns32(int rows, int ncol, const int* __restrict__ sel, const double2* __restrict__ v,
                                   float2* __restrict__ y) {
  const size_t n = (size_t)rows * ncol;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % rows), j = (int)(t / rows);
    const double2 a = v[(size_t)sel[j] * rows + i];
    y[t] = make_float2((float)a.x, (float)a.y);
  }
}

const cuComplex cOne = {1.f, 0.f};
const cuComplex cZero = {0.f, 0.f};
const cuComplex cMinusOne = {-1.f, 0.f};
inline cuComplex* Cf(float2* p) { return reinterpret_cast<cuComplex*>(p); }

// complex64 GEMM of the mixed subspace: plain CGEMM, or the Gauss three-product form (CGEMM3M)
// when HPSI_OPT_FP32_GEMM is 2
static int grid_of(size_t n) { return (int)std::min<size_t>(4096, (n + 255) / 256); }

cublasStatus_t cgemm32(const Context& c, cublasHandle_t h, cublasOperation_t ta, cublasOperation_t tb, int m, int n,
                       int k, const cuComplex* alpha, const cuComplex* A, int lda, const cuComplex* B, int ldb,
                       const cuComplex* beta, cuComplex* C, int ldc) {
  if (c.fp32_gemm == 2) return cublasCgemm3m(h, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
  return cublasCgemm(h, ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

// out[i] = sum over the nch chunks of part[c * stride + i], added in float64.
__global__ void k_sum_chunks(size_t n, int nch, size_t stride, const float2* __restrict__ part,
                             float2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double x = 0.0, y = 0.0;
    for (int ch = 0; ch < nch; ++ch) {
      const float2 v = part[ch * stride + i];
      x += v.x;
      y += v.y;
    }
    out[i] = make_float2((float)x, (float)y);
  }
}

// out[:, 0:nb] = A[:, 0:k] Y[0:k, 0:nb] for the tall A (ld npw).  A float32 GEMM accumulates its
// rounding error along k; with HPSI_OPT_RITZ_SPLIT the k range is cut into ceil(k / 128) (at most 8)
// equal chunks, each a float32 GEMM, and the chunk products are added in float64, so the error grows
// with the chunk length instead of k.  out must not overlap A or Y.
static int tall_gemm32(Context& c, DavHandles& h, int npw, int nb, int k, const float2* A, const float2* Y, int ldy,
                       float2* out) {
  DavWork& w = h.wk;
  const int nch = c.ritz_split ? std::min(8, (k + 127) / 128) : 1;
  if (nch <= 1) {
    BCK(cgemm32(c, h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nb, k, &cOne, reinterpret_cast<const cuComplex*>(A), npw,
                reinterpret_cast<const cuComplex*>(Y), ldy, &cZero, Cf(out), npw),
        "cgemm tall");
    return HPSI_OK;
  }
  const int kc = (k + nch - 1) / nch, nfull = k / kc, rem = k - nfull * kc;
  const int nparts = nfull + (rem > 0);
  const size_t stride = (size_t)npw * nb, need = stride * nparts;
  if (need > w.part_cap) {
    cudaFree(w.part32);
    w.part32 = nullptr;
    w.part_cap = 0;
    if (cudaMalloc((void**)&w.part32, sizeof(float2) * need) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, HPSI_ENOMEM, "davidson_solve: chunk-product allocation failed");
    }
    w.part_cap = need;
  }
  const cuComplex* a = reinterpret_cast<const cuComplex*>(A);
  const cuComplex* y = reinterpret_cast<const cuComplex*>(Y);
  if (c.fp32_gemm == 2)
    BCK(cublasCgemm3mStridedBatched(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nb, kc, &cOne, a, npw, (long long)kc * npw, y,
                                    ldy, kc, &cZero, Cf(w.part32), npw, (long long)stride, nfull),
        "cgemm chunks");
  else
    BCK(cublasCgemmStridedBatched(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nb, kc, &cOne, a, npw, (long long)kc * npw, y,
                                  ldy, kc, &cZero, Cf(w.part32), npw, (long long)stride, nfull),
        "cgemm chunks");
  if (rem > 0)
    BCK(cgemm32(c, h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nb, rem, &cOne, a + (size_t)nfull * kc * npw, npw,
                y + (size_t)nfull * kc, ldy, &cZero, Cf(w.part32 + (size_t)nfull * stride), npw),
        "cgemm chunk tail");
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_sum_chunks<<<grid_of(stride), 256, 0, c.stream>>>(stride, nparts, stride,
                                                                                       w.part32, out)));
  return HPSI_OK;
}

}  // namespace


// H applied to nb float32 vectors x32 -> float32 hx32, through the float64 staging buffers.
static int apply32(Context& c, DavWork& w, int ik, const float2* x32, float2* hx32, int nb) {
  const size_t n = (size_t)nb * w.npw;
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_cvt_32_64<<<grid_of(n), 256, 0, c.stream>>>(n, x32, w.in64)));
  int rc = apply_device(c, ik, w.in64, w.out64, nb);
  if (rc) return rc;
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_cvt_64_32<<<grid_of(n), 256, 0, c.stream>>>(n, w.out64, hx32)));
  return HPSI_OK;
}

// Orthonormalise the float32 block x[0:n] into out: Cholesky QR (float64 factor of the overlap) when
// the block is well conditioned, Cholesky QR twice when it is moderately conditioned (absolute
// threshold only), else canonically through the float64 eigen-decomposition of the overlap, where
// directions with overlap eigenvalue <= thr (relative to the largest if relative) drop.
// w.ovl32 = x^H x for the block x[0:n] (ld npw).
static int overlap32(Context& c, DavHandles& h, const float2* x, int n) {
  DavWork& w = h.wk;
  if (c.fp32_gemm == 4) return tc_inner32(c, w.tci, false, 0, x, n, x, n, w.npw, nullptr, w.ovl32, n);
  BCK(cgemm32(c, h.blas, CUBLAS_OP_C, CUBLAS_OP_N, n, n, w.npw, &cOne, reinterpret_cast<const cuComplex*>(x), w.npw,
              reinterpret_cast<const cuComplex*>(x), w.npw, &cZero, Cf(w.ovl32), n),
      "cgemm overlap");
  return HPSI_OK;
}

static int canonical_orth32(Context& c, DavHandles& h, const float2* x, int n, float2* out, int* nkeep, double thr,
                            bool relative) {
  DavWork& w = h.wk;
  const int npw = w.npw;
  int rc0 = overlap32(c, h, x, n);
  if (rc0) return rc0;
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_mat_32_to_64<<<(n * n + 255) / 256, 256, 0, c.stream>>>(n, n, w.ovl32, n, w.ovl, n)));
  // Cholesky QR (float64 factor of the overlap) when the block is well conditioned enough for a
  // float32 triangular solve (condition number of the factor below about 10)
  bool chol_ok = false;
  int rc = chol_overlap(c, h, n, relative ? 1e-6 : 1e-2, relative, &chol_ok);
  if (rc) return rc;
  if (chol_ok) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_mat_64_to_32<<<(n * n + 255) / 256, 256, 0, c.stream>>>(n, n, w.ovl, n, w.ovl32, n)));
    DCK(cudaMemcpyAsync(out, x, sizeof(float2) * (size_t)n * npw, cudaMemcpyDeviceToDevice, c.stream), "copy");
    BCK(cublasCtrsm(h.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, npw, n,
                    &cOne, Cf(w.ovl32), n, Cf(out), npw),
        "ctrsm");
    *nkeep = n;
    return HPSI_OK;
  }
  if (!relative) {
    // moderately conditioned correction block (factor condition below about 1e3): Cholesky QR twice,
    // the second pass on the (nearly orthonormal) result of the first
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_mat_32_to_64<<<(n * n + 255) / 256, 256, 0, c.stream>>>(n, n, w.ovl32, n, w.ovl, n)));
    bool loose_ok = false;
    rc = chol_overlap(c, h, n, 1e-6, false, &loose_ok);
    if (rc) return rc;
    if (loose_ok) {
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                  (k_mat_64_to_32<<<(n * n + 255) / 256, 256, 0, c.stream>>>(n, n, w.ovl, n, w.ovl32, n)));
      DCK(cudaMemcpyAsync(out, x, sizeof(float2) * (size_t)n * npw, cudaMemcpyDeviceToDevice, c.stream), "copy");
      BCK(cublasCtrsm(h.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, npw, n,
                      &cOne, Cf(w.ovl32), n, Cf(out), npw),
          "ctrsm");
      rc = overlap32(c, h, out, n);
      if (rc) return rc;
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                  (k_mat_32_to_64<<<(n * n + 255) / 256, 256, 0, c.stream>>>(n, n, w.ovl32, n, w.ovl, n)));
      bool second_ok = false;
      rc = chol_overlap(c, h, n, 1e-2, false, &second_ok);
      if (rc) return rc;
      if (second_ok) {
        HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                    (k_mat_64_to_32<<<(n * n + 255) / 256, 256, 0, c.stream>>>(n, n, w.ovl, n, w.ovl32, n)));
        BCK(cublasCtrsm(h.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, npw, n,
                        &cOne, Cf(w.ovl32), n, Cf(out), npw),
            "ctrsm");
        *nkeep = n;
        return HPSI_OK;
      }
    }
    // otherwise the overlap of x again, for its eigen-decomposition
    rc = overlap32(c, h, x, n);
    if (rc) return rc;
  }
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_mat_32_to_64<<<(n * n + 255) / 256, 256, 0, c.stream>>>(n, n, w.ovl32, n, w.ovl, n)));
  rc = small_eigh(c, h, w.ovl, n, n);
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
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_canon_scale32<<<(n * nk + 255) / 256, 256, 0, c.stream>>>(n, n, first, nk, w.evec, w.w, w.small32)));
  BCK(cgemm32(c, h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nk, n, &cOne, reinterpret_cast<const cuComplex*>(x), npw,
                  Cf(w.small32), n, &cZero, Cf(out), npw),
      "cgemm orthonormalise");
  return HPSI_OK;
}

// H_sub[0:rows, col0:col0+ncol] = phi32[0:rows]^H hphi32[col0:col0+ncol], stored in float64.
static int hsub_columns32(Context& c, DavHandles& h, int rows, int col0, int ncol) {
  DavWork& w = h.wk;
  const int npw = w.npw, mmax = w.mmax;
  if (c.fp32_gemm == 3)
    return w.sg.ah_b(c, h.blas, rows, ncol, npw, w.phi_split, w.phi32, npw, w.hphi32 + (size_t)col0 * npw, npw, 1.f,
                     0.f, nullptr, w.hsub + (size_t)col0 * mmax, mmax);
  if (c.fp32_gemm == 4)
    return tc_inner32(c, w.tci, true, mmax, w.phi32, rows, w.hphi32 + (size_t)col0 * npw, ncol, npw,
                      w.hsub + (size_t)col0 * mmax, nullptr, mmax);
  BCK(cgemm32(c, h.blas, CUBLAS_OP_C, CUBLAS_OP_N, rows, ncol, npw, &cOne, Cf(w.phi32), npw,
                  Cf(w.hphi32 + (size_t)col0 * npw), npw, &cZero, Cf(w.hcol32), mmax),
      "cgemm H_sub columns");
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_mat_32_to_64<<<(rows * ncol + 255) / 256, 256, 0, c.stream>>>(rows, ncol, w.hcol32, mmax,
                                                                                 w.hsub + (size_t)col0 * mmax, mmax)));
  return HPSI_OK;
}

// ---- the Davidson iteration, one loop for both precisions ----------------------------------------
// The loop below is written once; a precision policy supplies the basis arithmetic:
//   Fp64Ops  - complex128 basis, cuBLAS ZGEMMs and the float64 kernels; the eigenvalues are the
//              Ritz values of the last Rayleigh-Ritz step;
//   MixedOps - complex64 basis (float32 or emulated-float32 GEMMs), float64 small problems and
//              norms; hard locking, stall detection and a float64 Rayleigh quotient at exit.
// Both keep the basis orthonormal, restart from the wanted (or, thick, up to half the basis limit
// of the lowest) Ritz vectors and grow it by the orthonormalised preconditioned residuals of the
// unconverged bands (App. A.2.1).

struct Fp64Ops {
  using V = double2;
  static constexpr bool kMixed = false;
  Context& c;
  DavHandles& h;
  DavWork& w;
  const int ik, npw;
  Fp64Ops(Context& c_, DavHandles& h_, int ik_) : c(c_), h(h_), w(h_.wk), ik(ik_), npw(h_.wk.npw) {}
  V* phi() { return w.phi; }
  V* hphi() { return w.hphi; }
  V* psi() { return w.psi; }
  V* t() { return w.t; }
  void invalidate() {}
  // phi[0:N] <- the orthonormalised start
  int start(const double2* psio, int N, int* nk) { return canonical_orth(c, h, psio, N, w.phi, nk, 1e-12, true); }
  int apply(const V* x, V* hx, int nb) { return apply_device(c, ik, x, hx, nb); }
  // H_sub[0:rows, col0:col0+ncol] = phi[0:rows]^H hphi[col0:col0+ncol]
  int hsub(int rows, int col0, int ncol) {
    BCK(cublasZgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, rows, ncol, npw, &kOne, Z(w.phi), npw,
                    Z(w.hphi + (size_t)col0 * npw), npw, &kZero, Z(w.hsub + (size_t)col0 * w.mmax), w.mmax),
        "zgemm H_sub columns");
    return HPSI_OK;
  }
  // out = src[0:m] times the leading n columns of the reduced eigenvectors (ld m)
  int rotate(const V* src, int m, int n, V* out) {
    BCK(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, n, m, &kOne, Z(src), npw, Z(w.evec), m, &kZero, Z(out), npw),
        "zgemm Ritz vectors");
    return HPSI_OK;
  }
  // Ritz vectors psi = phi C[:, 0:NA], hpsi = hphi C[:, 0:NA]; residuals into t, norms into rnorm
  int ritz_residuals(int m, int NA) {
    int rc = rotate(w.phi, m, NA, w.psi);
    if (!rc) rc = rotate(w.hphi, m, NA, w.hpsi);
    if (rc) return rc;
    DCK(cudaMemcpyAsync(w.eps, w.w, sizeof(double) * NA, cudaMemcpyDeviceToDevice, c.stream), "eps copy");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_residual<<<NA, 256, 0, c.stream>>>(npw, w.psi, w.hpsi, w.eps, w.t, w.rnorm)));
    DCK(cudaGetLastError(), "residual kernel");
    return HPSI_OK;
  }
  // restart: phi, hphi <- the first keep Ritz vectors (psi, hpsi)
  int restart_copy(int keep) {
    DCK(cudaMemcpyAsync(w.phi, w.psi, sizeof(V) * (size_t)keep * npw, cudaMemcpyDeviceToDevice, c.stream), "restart copy");
    DCK(cudaMemcpyAsync(w.hphi, w.hpsi, sizeof(V) * (size_t)keep * npw, cudaMemcpyDeviceToDevice, c.stream),
        "restart copy");
    return HPSI_OK;
  }
  // thick restart: phi, hphi <- phi, hphi times the reduced eigenvectors sel (the lowest keep here:
  // the float64 solve locks nothing)
  int restart_rotate(int m, int keep, const std::vector<int>& sel) {
    for (int j = 0; j < keep; ++j)
      if (sel[j] != j) return fail(c, HPSI_EINVAL, "davidson_solve: internal restart selection error");
    for (V* src : {w.phi, w.hphi}) {
      int rc = rotate(src, m, keep, w.rst);
      if (rc) return rc;
      DCK(cudaMemcpyAsync(src, w.rst, sizeof(V) * (size_t)keep * npw, cudaMemcpyDeviceToDevice, c.stream),
          "restart copy");
    }
    return HPSI_OK;
  }
  int precondition(int nc, int eshift, V* tnew) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_precondition<<<nc, 256, 0, c.stream>>>(npw, w.idx, w.t, c.probs[ik].d_hdiag,
                                                                              w.eps, c.opt_tau, eshift, tnew)));
    DCK(cudaGetLastError(), "precondition kernel");
    return HPSI_OK;
  }
  // tnew[0:nc] -= phi[0:m] (phi[0:m]^H tnew)
  int project(int m, int /*locked*/, int nc, V* tnew) {
    BCK(cublasZgemm(h.blas, CUBLAS_OP_C, CUBLAS_OP_N, m, nc, npw, &kOne, Z(w.phi), npw, Z(tnew), npw, &kZero,
                    Z(w.small), m),
        "zgemm projection");
    BCK(cublasZgemm(h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nc, m, &kMinusOne, Z(w.phi), npw, Z(w.small), m, &kOne,
                    Z(tnew), npw),
        "zgemm projection update");
    return HPSI_OK;
  }
  int norm2(int nc, const V* tnew) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_norm2<<<nc, 256, 0, c.stream>>>(npw, tnew, w.cn2)));
    return HPSI_OK;
  }
  int fallback(int ncol, V* tnew) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_fallback<<<ncol, 256, 0, c.stream>>>(npw, w.idx2, w.idx, w.t, w.rnorm, tnew)));
    DCK(cudaGetLastError(), "fallback kernel");
    return HPSI_OK;
  }
  int orth(const V* x, int n, int* nkeep) { return canonical_orth(c, h, x, n, w.t, nkeep, kDropAbs, false); }
  // eigenvalues: the last Ritz values; eigenvectors: the last Ritz vectors
  int finish(int N, int /*locked*/, double2* psio, std::vector<double>& ev, std::vector<double>& rn, double* eig_out,
             double* resnorm_out) {
    DCK(cudaMemcpyAsync(psio, w.psi, sizeof(V) * (size_t)N * npw, cudaMemcpyDeviceToDevice, c.stream),
        "eigenvector copy");
    DCK(cudaMemcpyAsync(ev.data(), w.eps, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream), "eig copy");
    DCK(cudaStreamSynchronize(c.stream), "davidson end");
    for (int i = 0; i < N; ++i) {
      eig_out[i] = ev[i];
      if (resnorm_out) resnorm_out[i] = rn[i];
    }
    return HPSI_OK;
  }
  // the locked-vector and refresh operations exist only in the mixed form
  int lock(int, int, const int*) { return HPSI_OK; }
  int restart_gather(int, const std::vector<int>&) { return fail(c, HPSI_EINVAL, "davidson_solve: no locking in float64"); }
  int refresh(int, int) { return HPSI_OK; }
  int keep_active(int) { return HPSI_OK; }
};

struct MixedOps {
  using V = float2;
  static constexpr bool kMixed = true;
  Context& c;
  DavHandles& h;
  DavWork& w;
  const int ik, npw;
  const bool tc;   // subspace GEMMs through the bf16-split tensor-core products
  MixedOps(Context& c_, DavHandles& h_, int ik_)
      : c(c_), h(h_), w(h_.wk), ik(ik_), npw(h_.wk.npw), tc(c_.fp32_gemm == 3) {}
  // subspace GEMMs: float32 on the CUDA cores, or float32 emulated with bf16 tensor-core products
  // (cuBLAS math mode, restored by the destructor)
  int setup() {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_cvt_d2f<<<(npw + 255) / 256, 256, 0, c.stream>>>(npw, c.probs[ik].d_hdiag, w.hdiag32)));
    BCK(cublasSetMathMode(h.blas, c.fp32_gemm == 1 ? CUBLAS_FP32_EMULATED_BF16X9_MATH : CUBLAS_DEFAULT_MATH),
        "cublasSetMathMode");
    if (c.fp32_gemm == 1) {
      BCK(cublasSetEmulationStrategy(h.blas, CUBLAS_EMULATION_STRATEGY_EAGER), "cublasSetEmulationStrategy");
      // finite operands (a NaN would surface in the float64 residual norms): no special-value passes
      BCK(cublasSetEmulationSpecialValuesSupport(h.blas, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_NONE),
          "cublasSetEmulationSpecialValuesSupport");
    }
    invalidate();
    return HPSI_OK;
  }
  ~MixedOps() {
    cublasSetMathMode(h.blas, CUBLAS_DEFAULT_MATH);
    cublasSetEmulationSpecialValuesSupport(h.blas, CUDA_EMULATION_SPECIAL_VALUES_SUPPORT_DEFAULT);
  }
  V* phi() { return w.phi32; }
  V* hphi() { return w.hphi32; }
  V* psi() { return w.psi32; }
  V* t() { return w.t32; }
  // the cached bf16 splits of the basis are stale once its rows change
  void invalidate() {
    w.phi_split.invalidate();
    w.hphi_split.invalidate();
    w.tci.invalidate();
  }
  int start(const double2* psio, int N, int* nk) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_cvt_64_32<<<grid_of((size_t)N * npw), 256, 0, c.stream>>>((size_t)N * npw, psio, w.t32)));
    return canonical_orth32(c, h, w.t32, N, w.phi32, nk, 1e-12, true);
  }
  int apply(const V* x, V* hx, int nb) { return apply32(c, w, ik, x, hx, nb); }
  int hsub(int rows, int col0, int ncol) { return hsub_columns32(c, h, rows, col0, ncol); }
  int ritz_residuals(int m, int NA) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_mat_64_to_32<<<(m * NA + 255) / 256, 256, 0, c.stream>>>(m, NA, w.evec, m, w.small32, m)));
    int rc;
    if (tc) {
      rc = w.sg.a_b(c, h.blas, npw, NA, m, w.phi_split, w.phi32, npw, w.small32, m, 1.f, 0.f, w.psi32, npw);
      if (!rc) rc = w.sg.a_b(c, h.blas, npw, NA, m, w.hphi_split, w.hphi32, npw, w.small32, m, 1.f, 0.f, w.hpsi32, npw);
    } else {
      rc = tall_gemm32(c, h, npw, NA, m, w.phi32, w.small32, m, w.psi32);
      if (!rc) rc = tall_gemm32(c, h, npw, NA, m, w.hphi32, w.small32, m, w.hpsi32);
    }
    if (rc) return rc;
    DCK(cudaMemcpyAsync(w.eps, w.w, sizeof(double) * NA, cudaMemcpyDeviceToDevice, c.stream), "eps copy");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_residual32<<<NA, 1024, 0, c.stream>>>(npw, w.psi32, w.hpsi32, w.eps, w.t32, w.rnorm)));
    return HPSI_OK;
  }
  // the nl converged Ritz vectors sel (device list in idx2) join lock32 after the locked ones
  int lock(int locked, int nl, const int* sel) {
    DCK(cudaMemcpyAsync(w.idx2, sel, sizeof(int) * nl, cudaMemcpyHostToDevice, c.stream), "lock index copy");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_gather_rows32<<<nl, 256, 0, c.stream>>>(
                                        npw, w.idx2, w.psi32, w.lock32 + (size_t)locked * npw, nullptr, nullptr)));
    return HPSI_OK;
  }
  int restart_copy(int keep) {
    const size_t b = sizeof(V) * (size_t)keep * npw;
    DCK(cudaMemcpyAsync(w.phi32, w.psi32, b, cudaMemcpyDeviceToDevice, c.stream), "restart copy");
    DCK(cudaMemcpyAsync(w.hphi32, w.hpsi32, b, cudaMemcpyDeviceToDevice, c.stream), "restart copy");
    return HPSI_OK;
  }
  // restart from Ritz vectors already formed in psi32 / hpsi32, selected by sel
  int restart_gather(int keep, const std::vector<int>& sel) {
    DCK(cudaMemcpyAsync(w.sel, sel.data(), sizeof(int) * keep, cudaMemcpyHostToDevice, c.stream), "restart index copy");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_gather_rows32<<<keep, 256, 0, c.stream>>>(npw, w.sel, w.psi32, w.phi32, w.hpsi32, w.hphi32)));
    return HPSI_OK;
  }
  // thick restart: phi32 and hphi32 times the selected reduced eigenvectors
  int restart_rotate(int m, int keep, const std::vector<int>& sel) {
    DCK(cudaMemcpyAsync(w.sel, sel.data(), sizeof(int) * keep, cudaMemcpyHostToDevice, c.stream), "restart index copy");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_select_columns32<<<grid_of((size_t)m * keep), 256, 0, c.stream>>>(
                                        m, keep, w.sel, w.evec, w.ysub32)));
    for (int pass = 0; pass < 2; ++pass) {
      float2* src = pass == 0 ? w.phi32 : w.hphi32;
      int rc;
      if (tc)
        rc = w.sg.a_b(c, h.blas, npw, keep, m, pass == 0 ? w.phi_split : w.hphi_split, src, npw, w.ysub32, m, 1.f,
                      0.f, w.rst32, npw);
      else
        rc = tall_gemm32(c, h, npw, keep, m, src, w.ysub32, m, w.rst32);
      if (rc) return rc;
      DCK(cudaMemcpyAsync(src, w.rst32, sizeof(V) * (size_t)keep * npw, cudaMemcpyDeviceToDevice, c.stream),
          "restart copy");
    }
    return HPSI_OK;
  }
  // H applied afresh to the keep restart vectors (replacing stored products that drifted)
  int refresh(int keep, int N) {
    for (int b = 0; b < keep; b += N) {
      const int rc = apply32(c, w, ik, w.phi32 + (size_t)b * npw, w.hphi32 + (size_t)b * npw, std::min(N, keep - b));
      if (rc) return rc;
    }
    return HPSI_OK;
  }
  // psi32 keeps the na active Ritz vectors in the new numbering for an exit before the next step
  int keep_active(int na) {
    DCK(cudaMemcpyAsync(w.psi32, w.phi32, sizeof(V) * (size_t)na * npw, cudaMemcpyDeviceToDevice, c.stream),
        "active copy");
    return HPSI_OK;
  }
  int precondition(int nc, int eshift, V* tnew) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_precondition32<<<nc, 1024, 0, c.stream>>>(npw, w.idx, w.t32, w.hdiag32, w.eps,
                                                                                c.opt_tau, eshift, tnew)));
    return HPSI_OK;
  }
  // Block Gram-Schmidt against [lock32, phi32] (the locked vectors are orthogonal to the basis, so
  // projecting them out first is the same as projecting out the union in one block).
  int project(int m, int locked, int nc, V* tnew) {
    if (locked > 0) {
      BCK(cgemm32(c, h.blas, CUBLAS_OP_C, CUBLAS_OP_N, locked, nc, npw, &cOne, Cf(w.lock32), npw, Cf(tnew), npw,
                  &cZero, Cf(w.small32), locked),
          "cgemm lock projection");
      BCK(cgemm32(c, h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nc, locked, &cMinusOne, Cf(w.lock32), npw, Cf(w.small32),
                  locked, &cOne, Cf(tnew), npw),
          "cgemm lock projection update");
    }
    if (tc) {
      int r = w.sg.ah_b(c, h.blas, m, nc, npw, w.phi_split, w.phi32, npw, tnew, npw, 1.f, 0.f, w.small32, nullptr, m);
      if (!r) r = w.sg.a_b(c, h.blas, npw, nc, m, w.phi_split, w.phi32, npw, w.small32, m, -1.f, 1.f, tnew, npw);
      return r;
    }
    if (c.fp32_gemm == 4) {
      const int r = tc_inner32(c, w.tci, true, w.mmax, w.phi32, m, tnew, nc, npw, nullptr, w.small32, m);
      if (r) return r;
    } else {
      BCK(cgemm32(c, h.blas, CUBLAS_OP_C, CUBLAS_OP_N, m, nc, npw, &cOne, Cf(w.phi32), npw, Cf(tnew), npw, &cZero,
                  Cf(w.small32), m),
          "cgemm projection");
    }
    BCK(cgemm32(c, h.blas, CUBLAS_OP_N, CUBLAS_OP_N, npw, nc, m, &cMinusOne, Cf(w.phi32), npw, Cf(w.small32), m, &cOne,
                Cf(tnew), npw),
        "cgemm projection update");
    return HPSI_OK;
  }
  int norm2(int nc, const V* tnew) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_norm2_32<<<nc, 1024, 0, c.stream>>>(npw, tnew, w.cn2)));
    return HPSI_OK;
  }
  int fallback(int ncol, V* tnew) {
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_fallback32<<<ncol, 1024, 0, c.stream>>>(npw, w.idx2, w.idx, w.t32, w.rnorm, tnew)));
    return HPSI_OK;
  }
  int orth(const V* x, int n, int* nkeep) { return canonical_orth32(c, h, x, n, w.t32, nkeep, kDropAbs, false); }
  // float64 Rayleigh quotients of the Ritz vectors (locked ones first) with a fresh H|psi>, by
  // default with float64 projections and D: the eigenvalue error is then second order in the
  // eigenvector error left by the mixed iterations.  Bands are returned in ascending order.
  int finish(int N, int locked, double2* psio, std::vector<double>& ev, std::vector<double>& rn, double* eig_out,
             double* resnorm_out) {
    const size_t n = (size_t)N * npw, nl = (size_t)locked * npw;
    if (locked > 0)
      HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_cvt_32_64<<<grid_of(nl), 256, 0, c.stream>>>(nl, w.lock32, w.in64)));
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
                (k_cvt_32_64<<<grid_of(n - nl), 256, 0, c.stream>>>(n - nl, w.psi32, w.in64 + nl)));
    final_precision_begin(c);
    int rc = apply_device(c, ik, w.in64, w.out64, N);
    final_precision_end(c);
    if (rc) return rc;
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_rayleigh<<<N, 1024, 0, c.stream>>>(npw, w.in64, w.out64, w.eps, w.rnorm)));
    DCK(cudaMemcpyAsync(ev.data(), w.eps, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream), "eig copy");
    DCK(cudaMemcpyAsync(rn.data(), w.rnorm, sizeof(double) * N, cudaMemcpyDeviceToHost, c.stream), "norm copy");
    DCK(cudaStreamSynchronize(c.stream), "davidson end");
    rc = check_device_error(c);
    if (rc) return rc;
    std::vector<int> perm(N);
    for (int i = 0; i < N; ++i) perm[i] = i;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return ev[a] < ev[b]; });
    DCK(cudaMemcpyAsync(w.idx, perm.data(), sizeof(int) * N, cudaMemcpyHostToDevice, c.stream), "perm copy");
    HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_gather_rows<<<N, 256, 0, c.stream>>>(npw, w.idx, w.in64, psio)));
    DCK(cudaStreamSynchronize(c.stream), "davidson end");
    for (int i = 0; i < N; ++i) {
      eig_out[i] = ev[perm[i]];
      if (resnorm_out) resnorm_out[i] = rn[perm[i]];
    }
    return HPSI_OK;
  }
};

template <class Ops>
static int davidson_loop(Context& c, DavHandles& h, Ops& ops, int N, double tol, int maxiter, double2* psio,
                         double* eig_out, int* iters_out, double* resnorm_out) {
  using V = typename Ops::V;
  DavWork& w = h.wk;
  const int npw = w.npw, mmax = w.mmax;
  const size_t vb = sizeof(V) * (size_t)npw;
  // phi[0:N] <- orthonormalised initial guess, hphi = H phi, H_sub = phi^H hphi
  int nk = 0;
  int rc = ops.start(psio, N, &nk);
  if (rc) return rc;
  if (nk < N) return fail(c, HPSI_EINVAL, "davidson_solve: initial guess is linearly dependent");
  rc = ops.apply(ops.phi(), ops.hphi(), N);
  if (rc) return rc;
  int m = N;
  rc = ops.hsub(m, 0, m);
  if (rc) return rc;
  std::vector<double> rn(N), ev(N), cn;
  std::vector<int> uidx(N), lsel, asel, col;
  int it = 0;
  bool converged = false;
  // Hard locking (mixed form only): the first kL bands are frozen in lock32; the reduced basis
  // phi[0:m] spans only the active part of the search space (orthogonal to lock32) and the
  // Rayleigh-Ritz step asks it for the NA = N - kL lowest pairs.  Without locking kL stays 0.
  int kL = 0;
  // Ritz vectors a restart keeps: the active ones, or with thick restart up to half the basis limit.
  // In the mixed form a thick-restarted vector is a float32 rotation of the basis whose stored
  // H|phi> is the same rotation of the stored products; the two drift apart by rounding amplified
  // by the largest eigenvalue of H, so a solve whose largest residual stops falling (kStall
  // iterations without a 10% drop) goes on with plain restarts, then with H applied afresh.
  bool thick = c.thick_restart != 0;
  bool refresh = false;
  int stall = 0;
  double best = INFINITY;
  auto basis_limit = [&](int locked) { return locked > 0 ? std::min(mmax, c.lock_basis * (N - locked)) : mmax; };
  auto restart_size = [&](int locked, int m_avail) {
    const int na = N - locked;
    return thick ? std::min(m_avail, std::min(w.kmax, std::max(na, basis_limit(locked) / 2))) : na;
  };
  for (;;) {
    const int NA = N - kL;
    const int mlim = basis_limit(kL);
    // a restart is certain once m + NA > mlim unless bands converge; solve for its kept vectors now
    int nev = NA;
    if (m + NA > mlim) nev = std::max(NA, restart_size(kL, m));
    rc = lowest_eigh(c, h, w.hsub, mmax, m, nev);
    if (rc) return rc;
    rc = ops.ritz_residuals(m, NA);
    if (rc) return rc;
    DCK(cudaMemcpyAsync(rn.data(), w.rnorm, sizeof(double) * NA, cudaMemcpyDeviceToHost, c.stream), "norm copy");
    DCK(cudaStreamSynchronize(c.stream), "davidson iteration");
    rc = check_device_error(c);
    if (rc) return rc;
    int nc = 0;
    double rmax = 0.0;
    for (int i = 0; i < NA; ++i) {
      rmax = std::max(rmax, rn[i]);
      if (!(rn[i] <= tol)) uidx[nc++] = i;
    }
    if (nc == 0) {
      converged = true;
      break;
    }
    if (it >= maxiter) break;
    ++it;
    lsel.clear();
    if constexpr (Ops::kMixed) {
      if (rmax < 0.9 * best) {
        best = rmax;
        stall = 0;
      } else if (++stall >= kStall) {
        stall = 0;
        if (thick) thick = false;
        else refresh = true;
      }
      // Lock: converged Ritz vectors move to lock32.  t, eps and rnorm keep this iteration's
      // numbering, which uidx indexes.
      if (c.locking) {
        if (c.locking == 1) {
          while ((int)lsel.size() < NA && rn[lsel.size()] <= tol) lsel.push_back((int)lsel.size());
        } else {
          for (int i = 0; i < NA; ++i)
            if (rn[i] <= tol) lsel.push_back(i);
        }
        if ((int)lsel.size() < std::max(1, (int)std::ceil(c.lock_batch * NA))) lsel.clear();
      }
    }
    const int nl = (int)lsel.size();
    if (nl > 0 || m + nc > mlim || refresh) {
      if (nl > 0) {
        rc = ops.lock(kL, nl, lsel.data());
        if (rc) return rc;
      }
      // restart from the lowest Ritz vectors that are not locked
      const int kL2 = kL + nl, na = N - kL2;
      const int keep = restart_size(kL2, m - nl);
      asel.clear();
      for (int i = 0, j = 0; i < m && (int)asel.size() < keep; ++i) {
        if (j < nl && lsel[j] == i) {
          ++j;
          continue;
        }
        asel.push_back(i);
      }
      if (asel.back() < NA) {
        // every kept vector is an active Ritz vector already formed in psi / hpsi
        rc = nl == 0 ? ops.restart_copy(keep) : ops.restart_gather(keep, asel);
      } else {
        // thick restart: the kept Ritz vectors are phi and hphi times the selected reduced eigenvectors
        if (asel.back() >= nev) {
          rc = lowest_eigh(c, h, w.hsub, mmax, m, asel.back() + 1);
          if (rc) return rc;
        }
        rc = ops.restart_rotate(m, keep, asel);
      }
      if (rc) return rc;
      if (refresh) {
        rc = ops.refresh(keep, N);
        if (rc) return rc;
        refresh = false;
      }
      if (nl > 0) {
        rc = ops.keep_active(na);
        if (rc) return rc;
      }
      kL = kL2;
      ops.invalidate();
      m = keep;
      rc = ops.hsub(m, 0, m);
      if (rc) return rc;
    }
    DCK(cudaMemcpyAsync(w.idx, uidx.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, c.stream), "index copy");
    // corrections into phi[m : m+nc] (t holds the residuals)
    V* tnew = ops.phi() + (size_t)m * npw;
    rc = ops.precondition(nc, c.opt_shift == 1 ? NA - 1 : -1, tnew);
    if (rc) return rc;
    cn.resize(nc);
    auto norms = [&]() -> int {
      int r = ops.norm2(nc, tnew);
      if (r) return r;
      DCK(cudaMemcpyAsync(cn.data(), w.cn2, sizeof(double) * nc, cudaMemcpyDeviceToHost, c.stream), "norm copy");
      DCK(cudaStreamSynchronize(c.stream), "correction norms");
      return HPSI_OK;
    };
    // Block Gram-Schmidt against the basis.  The corrections enter with unit norm.  One pass leaves
    // them orthogonal to the basis up to rounding relative to their norm before it; a second pass
    // only helps a column that the first cancelled (kept less than kReorth of its squared norm), so
    // with HPSI_OPT_REORTH_TEST it runs only then.
    for (int round = 0; round < 2; ++round) {
      rc = ops.project(m, kL, nc, tnew);
      if (rc) return rc;
      bool second = round == 1 || !c.reorth_test;
      if (!second) {
        rc = norms();
        if (rc) return rc;
        for (int j = 0; j < nc; ++j)
          if (!(cn[j] >= kReorth)) second = true;
      }
      if (second) {
        rc = ops.project(m, kL, nc, tnew);
        if (rc) return rc;
      }
      if (round == 1) break;
      if (second) {
        rc = norms();
        if (rc) return rc;
      }
      // corrections that lie in the basis are replaced by their raw residuals
      col.clear();
      for (int j = 0; j < nc; ++j)
        if (!(cn[j] >= kCollapse)) col.push_back(j);
      if (col.empty()) break;
      DCK(cudaMemcpyAsync(w.idx2, col.data(), sizeof(int) * col.size(), cudaMemcpyHostToDevice, c.stream),
          "index copy");
      rc = ops.fallback((int)col.size(), tnew);
      if (rc) return rc;
    }
    // orthonormalise the block itself (t is free now: the residuals were consumed)
    int nkeep = 0;
    rc = ops.orth(tnew, nc, &nkeep);
    if (rc) return rc;
    if (nkeep == 0) break;   // nothing new can be added: the residuals lie in the basis up to rounding
    DCK(cudaMemcpyAsync(tnew, ops.t(), vb * nkeep, cudaMemcpyDeviceToDevice, c.stream), "basis copy");
    rc = ops.apply(tnew, ops.hphi() + (size_t)m * npw, nkeep);
    if (rc) return rc;
    // new columns of H_sub: phi[0:m+nkeep]^H hphi[m:m+nkeep] (the upper triangle is what is read)
    rc = ops.hsub(m + nkeep, m, nkeep);
    if (rc) return rc;
    m += nkeep;
  }
  rc = ops.finish(N, kL, psio, ev, rn, eig_out, resnorm_out);
  if (rc) return rc;
  if (iters_out) *iters_out = it;
  if (!converged) return fail(c, HPSI_ENOTCONV, "davidson_solve: not converged within maxiter");
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
  const bool mixed = c.precision == HPSI_MIXED;
  int rc = alloc_work(c, *h, p.npw, nbnd, mixed);
  if (rc) return rc;
  if (!mixed) {
    Fp64Ops ops(c, *h, ik);
    return davidson_loop(c, *h, ops, nbnd, tol, maxiter, psio, eig_out, iters_out, resnorm_out);
  }
  MixedOps ops(c, *h, ik);
  rc = ops.setup();
  if (rc) return rc;
  return davidson_loop(c, *h, ops, nbnd, tol, maxiter, psio, eig_out, iters_out, resnorm_out);
}

}  // namespace hpsi
