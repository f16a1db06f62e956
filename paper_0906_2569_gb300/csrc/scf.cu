// Self-consistency loop around the eigensolver (paper App. A.1), on the GPU.
//
// The Kohn-Sham problem is a fixed point in the density: rho_in gives V = V_ext + V_H[rho_in] +
// V_xc[rho_in], the lowest orbitals of H[V] give rho_out = sum_i f_i |psi_i|^2, and the next input
// is the combination of the last few inputs whose combined residual rho_out - rho_in has the
// smallest scf norm, plus a fraction of that residual.  The scf norm is the Hartree energy of the
// density difference, ||d rho||^2 = 4 pi Omega sum_{G != 0} |d rho(G)|^2 / G^2 (= 2 E_H[d rho]).
//
// Conventions (those of H|psi>): psi(r_j) = sum_G psi(G) e^{i(k+G).r_j} with sum_G |psi(G)|^2 = 1,
// so the density on the grid is rho(r_j) = sum_i f_i |psi_i(r_j)|^2 / (Omega <psi_i|psi_i>) (each
// orbital normalised, so the charge is exact whatever the eigensolver's rounding); a grid function's
// Fourier components are a(G) = N_r^-1 sum_j a(r_j) e^{-iG.r_j}; V_H(G) = 4 pi rho(G) / G^2 with
// V_H(G = 0) = 0 (neutralising background); LDA is Slater exchange plus the Perdew-Zunger fit of
// the Ceperley-Alder correlation of the unpolarised gas; the nocc lowest bands hold two electrons
// each.  Mixing is the Anderson form of the scf-norm minimisation over the last nmix pairs with a
// step beta along the optimal residual.  Energies (no ion-ion term):
//   E     = sum_i f_i eps_i - int rho_out V_Hxc[rho_in] + E_Hxc[rho_out]
//   E_HWF = sum_i f_i eps_i - int rho_in  V_Hxc[rho_in] + E_Hxc[rho_in]   (Harris-Weinert-Foulkes)
//
// Every grid step runs in the kernels below: the density from the orbitals' inverse transforms
// (local_kernels.cu), full-box line FFTs of the grid functions (the warp line transforms of the
// local kernels), the Hartree and LDA terms, the scf-norm inner products and the mixing updates.
// The host solves the mixing's small least-squares system (at most nmix - 1 unknowns).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "hpsi_internal.h"
#include "box_fft.cuh"

namespace hpsi {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kRedBlocks = 304;        // partial sums per reduction (2 per SM), summed on the host in order
constexpr int kMaxMix = 16;

struct Recip {
  double b[9];
};

// signed frequency of index j on an axis of n points (numpy's fftfreq order)
__device__ __forceinline__ int signed_freq(int j, int n) { return 2 * j < n ? j : j - n; }

__device__ __forceinline__ double block_sum(double s) {
  __shared__ double red[33];
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

__global__ void k_real_to_box(size_t n, const double* __restrict__ a, const double* __restrict__ b, double2* __restrict__ box) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    box[i] = make_double2(b ? a[i] - b[i] : a[i], 0.0);
}

// box holds sum_j a(r_j) e^{-iG.r_j}: it becomes a(G) (scaled by 1/N_r) or, with write set,
// 4 pi a(G) / G^2 (V_H(G)); partial[block] receives sum 4 pi |a(G)|^2 / G^2 over G != 0.
__global__ void __launch_bounds__(256) k_hartree_g(double2* __restrict__ box, int n1, int n2, int n3, Recip rc,
                                                   double inv_nr, int write, double* __restrict__ partial) {
  const size_t n = (size_t)n1 * n2 * n3;
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int j1 = (int)(i % n1), j2 = (int)((i / n1) % n2), j3 = (int)(i / ((size_t)n1 * n2));
    const double m1 = signed_freq(j1, n1), m2 = signed_freq(j2, n2), m3 = signed_freq(j3, n3);
    const double gx = m1 * rc.b[0] + m2 * rc.b[3] + m3 * rc.b[6];
    const double gy = m1 * rc.b[1] + m2 * rc.b[4] + m3 * rc.b[7];
    const double gz = m1 * rc.b[2] + m2 * rc.b[5] + m3 * rc.b[8];
    const double g2 = gx * gx + gy * gy + gz * gz;
    const double2 v = make_double2(box[i].x * inv_nr, box[i].y * inv_nr);
    const double f = g2 > 1e-12 ? 4.0 * kPi / g2 : 0.0;
    acc += f * (v.x * v.x + v.y * v.y);
    box[i] = write ? make_double2(f * v.x, f * v.y) : v;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// the scf-norm weight 4 pi Omega / G^2 of each box point (0 at G = 0)
__global__ void k_norm_weight(int n1, int n2, int n3, Recip rc, double omega, double* __restrict__ w) {
  const size_t n = (size_t)n1 * n2 * n3;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int j1 = (int)(i % n1), j2 = (int)((i / n1) % n2), j3 = (int)(i / ((size_t)n1 * n2));
    const double m1 = signed_freq(j1, n1), m2 = signed_freq(j2, n2), m3 = signed_freq(j3, n3);
    const double gx = m1 * rc.b[0] + m2 * rc.b[3] + m3 * rc.b[6];
    const double gy = m1 * rc.b[1] + m2 * rc.b[4] + m3 * rc.b[7];
    const double gz = m1 * rc.b[2] + m2 * rc.b[5] + m3 * rc.b[8];
    const double g2 = gx * gx + gy * gy + gz * gz;
    w[i] = g2 > 1e-12 ? 4.0 * kPi * omega / g2 : 0.0;
  }
}

// V_H(r) = Re(box) (after the inverse transform) plus V_xc, and the energy density of exchange and
// correlation: Slater exchange, Perdew-Zunger correlation (zero where rho <= 1e-30).
// vtot = vext + V_H + V_xc; vhxc = V_H + V_xc; partial: sum rho eps_xc.
__global__ void __launch_bounds__(256) k_lda(size_t n, const double* __restrict__ rho, const double2* __restrict__ box,
                                             const double* __restrict__ vext, double* __restrict__ vhxc,
                                             double* __restrict__ vtot, double* __restrict__ partial) {
  const double gam = -0.1423, be1 = 1.0529, be2 = 0.3334, A = 0.0311, B = -0.048, C = 0.0020, D = -0.0116;
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double r = rho[i];
    double exc = 0.0, vxc = 0.0;
    if (r > 1e-30) {
      const double rs = cbrt(3.0 / (4.0 * kPi * r));
      const double ex = -0.75 * cbrt(3.0 * r / kPi);
      const double vx = 4.0 / 3.0 * ex;
      double ec, vc;
      if (rs >= 1.0) {
        const double s = sqrt(rs);
        const double den = 1.0 + be1 * s + be2 * rs;
        ec = gam / den;
        vc = ec * (1.0 + 7.0 / 6.0 * be1 * s + 4.0 / 3.0 * be2 * rs) / den;
      } else {
        const double lx = log(rs);
        ec = A * lx + B + C * rs * lx + D * rs;
        vc = A * lx + (B - A / 3.0) + 2.0 / 3.0 * C * rs * lx + (2.0 * D - C) / 3.0 * rs;
      }
      exc = ex + ec;
      vxc = vx + vc;
    }
    acc += r * exc;
    const double v = box[i].x + vxc;
    vhxc[i] = v;
    vtot[i] = vext[i] + v;
  }
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// partial[block] = sum a[i] b[i]
__global__ void __launch_bounds__(256) k_dot(size_t n, const double* __restrict__ a, const double* __restrict__ b,
                                             double* __restrict__ partial) {
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += a[i] * (b ? b[i] : 1.0);
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// partial[block] = sum w[i] Re(conj(a[i]) b[i])
__global__ void __launch_bounds__(256) k_wdot(size_t n, const double2* __restrict__ a, const double2* __restrict__ b,
                                              const double* __restrict__ w, double* __restrict__ partial) {
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += w[i] * (a[i].x * b[i].x + a[i].y * b[i].y);
  acc = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// y = a x + b y (real or, through the element count, interleaved complex)
__global__ void k_axpby(size_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void k_sub(size_t n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

// occ[b] = f / (Omega <psi_b|psi_b>): the density of the normalised orbital; one CTA per band
__global__ void __launch_bounds__(256) k_occ_weights(int npw, const double2* __restrict__ psi, double f_over_omega,
                                                     double* __restrict__ occ) {
  const double2* x = psi + (size_t)blockIdx.x * npw;
  double s = 0.0;
  for (int g = threadIdx.x; g < npw; g += blockDim.x) s = fma(x[g].x, x[g].x, fma(x[g].y, x[g].y, s));
  s = block_sum(s);
  if (threadIdx.x == 0) occ[blockIdx.x] = f_over_omega / s;
}

int grid_for(size_t n) { return (int)std::min<size_t>(4096, (n + 255) / 256); }

}  // namespace

struct ScfWork {
  size_t nr = 0;
  int nmix = 0;
  double2* box = nullptr;
  double* wgt = nullptr;       // scf-norm weights
  double* vext = nullptr;
  double* vhxc = nullptr;
  double* vtot = nullptr;
  double* rho_in = nullptr;
  double* rho_out = nullptr;
  double* xin = nullptr;       // [nmix][nr] past inputs
  double* res = nullptr;       // [nmix][nr] past residuals
  double2* rhat = nullptr;     // [nmix][nr] their Fourier components
  double* tmp = nullptr;       // [nr]
  double* occ = nullptr;       // [nbnd] f_i / Omega
  double* partial = nullptr;   // [kRedBlocks]
  int occ_cap = 0;
};

static void free_scf(ScfWork& w) {
  cudaFree(w.box);
  for (double* p : {w.wgt, w.vext, w.vhxc, w.vtot, w.rho_in, w.rho_out, w.xin, w.res, w.tmp, w.occ, w.partial})
    cudaFree(p);
  cudaFree(w.rhat);
  w = ScfWork();
}

void scf_release(Context& c) {
  ScfWork* w = reinterpret_cast<ScfWork*>(c.scf);
  if (!w) return;
  free_scf(*w);
  delete w;
  c.scf = nullptr;
}

#define SCK(x, what)                                      \
  do {                                                    \
    cudaError_t e_ = (x);                                 \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

namespace {

class Scf {
 public:
  Scf(Context& c, int ik) : c_(c), ik_(ik), p_(c.probs[ik]) {
    nr_ = (size_t)p_.n[0] * p_.n[1] * p_.n[2];
    for (int i = 0; i < 9; ++i) rc_.b[i] = p_.recip[i];
    omega_ = std::fabs(p_.cell[0] * (p_.cell[4] * p_.cell[8] - p_.cell[5] * p_.cell[7]) -
                       p_.cell[1] * (p_.cell[3] * p_.cell[8] - p_.cell[5] * p_.cell[6]) +
                       p_.cell[2] * (p_.cell[3] * p_.cell[7] - p_.cell[4] * p_.cell[6]));
  }

  int alloc(int nmix, int nbnd);
  // box <- forward transform of a (- b), scaled to Fourier components; the scf-norm energy
  // sum 4 pi Omega |.|^2 / G^2 in *norm2 (nullable); with hartree, box <- V_H(G) then V_H(r).
  int transform(const double* a, const double* b, double* norm2, bool hartree);
  int hxc(const double* rho, double* ehxc);   // w.vhxc, w.vtot; E_H + E_xc
  int dot(const double* a, const double* b, double* out);
  int wdot(const double2* a, const double2* b, double* out);
  int run(int nocc, int nbnd, double tol, int maxiter, double2* psi, double* eig_out, double* energies,
          int* iters_out, double* norm2_out);

  ScfWork* w_ = nullptr;

 private:
  Context& c_;
  int ik_;
  const Problem& p_;
  size_t nr_;
  Recip rc_;
  double omega_;

  int sum_partials(double* out);
  int fft(int dir);
};

int Scf::alloc(int nmix, int nbnd) {
  Context& c = c_;
  ScfWork* w = reinterpret_cast<ScfWork*>(c.scf);
  if (!w) {
    w = new ScfWork();
    c.scf = w;
  }
  w_ = w;
  if (w->nr != nr_ || w->nmix != nmix) {
    free_scf(*w);
    auto al = [&](void** p, size_t bytes) -> bool {
      if (cudaMalloc(p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      return true;
    };
    const size_t r = sizeof(double) * nr_;
    bool ok = al((void**)&w->box, 2 * r) && al((void**)&w->wgt, r) && al((void**)&w->vext, r) &&
              al((void**)&w->vhxc, r) && al((void**)&w->vtot, r) && al((void**)&w->rho_in, r) &&
              al((void**)&w->rho_out, r) && al((void**)&w->xin, r * nmix) && al((void**)&w->res, r * nmix) &&
              al((void**)&w->rhat, 2 * r * nmix) && al((void**)&w->tmp, r) &&
              al((void**)&w->partial, sizeof(double) * kRedBlocks);
    if (!ok) {
      free_scf(*w);
      return fail(c, HPSI_ENOMEM, "hpsi_scf: device allocation failed");
    }
    w->nr = nr_;
    w->nmix = nmix;
  }
  if (w->occ_cap < nbnd) {
    cudaFree(w->occ);
    w->occ = nullptr;
    w->occ_cap = 0;
    if (cudaMalloc((void**)&w->occ, sizeof(double) * nbnd) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, HPSI_ENOMEM, "hpsi_scf: device allocation failed");
    }
    w->occ_cap = nbnd;
  }
  return HPSI_OK;
}

int Scf::sum_partials(double* out) {
  Context& c = c_;
  std::vector<double> h(kRedBlocks);
  SCK(cudaMemcpyAsync(h.data(), w_->partial, sizeof(double) * kRedBlocks, cudaMemcpyDeviceToHost, c.stream),
      "partial sums copy");
  SCK(cudaStreamSynchronize(c.stream), "partial sums");
  double s = 0.0;
  for (double v : h) s += v;
  *out = s;
  return HPSI_OK;
}

int Scf::fft(int dir) { return box_fft(c_, p_, w_->box, 1, dir, HPSI_K_SCF); }

int Scf::transform(const double* a, const double* b, double* norm2, bool hartree) {
  Context& c = c_;
  HPSI_LAUNCH(c, HPSI_K_SCF, (k_real_to_box<<<grid_for(nr_), 256, 0, c.stream>>>(nr_, a, b, w_->box)));
  int rc = fft(-1);
  if (rc) return rc;
  HPSI_LAUNCH(c, HPSI_K_SCF, (k_hartree_g<<<kRedBlocks, 256, 0, c.stream>>>(w_->box, p_.n[0], p_.n[1], p_.n[2], rc_,
                                                                            1.0 / (double)nr_, hartree ? 1 : 0,
                                                                            w_->partial)));
  SCK(cudaGetLastError(), "Hartree kernel");
  if (norm2) {
    double s = 0.0;
    rc = sum_partials(&s);
    if (rc) return rc;
    *norm2 = omega_ * s;
  }
  if (hartree) return fft(+1);
  return HPSI_OK;
}

int Scf::hxc(const double* rho, double* ehxc) {
  Context& c = c_;
  double eh2 = 0.0;
  int rc = transform(rho, nullptr, &eh2, true);   // box <- V_H(r) (imaginary part ~ rounding)
  if (rc) return rc;
  HPSI_LAUNCH(c, HPSI_K_SCF, (k_lda<<<kRedBlocks, 256, 0, c.stream>>>(nr_, rho, w_->box, w_->vext, w_->vhxc,
                                                                      w_->vtot, w_->partial)));
  SCK(cudaGetLastError(), "LDA kernel");
  double exc = 0.0;
  rc = sum_partials(&exc);
  if (rc) return rc;
  *ehxc = 0.5 * eh2 + omega_ * exc / (double)nr_;
  return HPSI_OK;
}

int Scf::dot(const double* a, const double* b, double* out) {
  Context& c = c_;
  HPSI_LAUNCH(c, HPSI_K_SCF, (k_dot<<<kRedBlocks, 256, 0, c.stream>>>(nr_, a, b, w_->partial)));
  SCK(cudaGetLastError(), "dot kernel");
  return sum_partials(out);
}

int Scf::wdot(const double2* a, const double2* b, double* out) {
  Context& c = c_;
  HPSI_LAUNCH(c, HPSI_K_SCF, (k_wdot<<<kRedBlocks, 256, 0, c.stream>>>(nr_, a, b, w_->wgt, w_->partial)));
  SCK(cudaGetLastError(), "weighted dot kernel");
  return sum_partials(out);
}

// Solve the k x k system A g = b (row-major) by Gaussian elimination with partial pivoting;
// false if a pivot is negligible (the caller then drops the oldest history entry).
static bool small_solve(int k, std::vector<double> A, std::vector<double> b, std::vector<double>* g) {
  double amax = 0.0;
  for (double v : A) amax = std::max(amax, std::fabs(v));
  for (int col = 0; col < k; ++col) {
    int piv = col;
    for (int r = col + 1; r < k; ++r)
      if (std::fabs(A[r * k + col]) > std::fabs(A[piv * k + col])) piv = r;
    if (!(std::fabs(A[piv * k + col]) > 1e-14 * amax)) return false;
    if (piv != col) {
      for (int j = 0; j < k; ++j) std::swap(A[col * k + j], A[piv * k + j]);
      std::swap(b[col], b[piv]);
    }
    for (int r = col + 1; r < k; ++r) {
      const double f = A[r * k + col] / A[col * k + col];
      for (int j = col; j < k; ++j) A[r * k + j] -= f * A[col * k + j];
      b[r] -= f * b[col];
    }
  }
  g->assign(k, 0.0);
  for (int r = k - 1; r >= 0; --r) {
    double s = b[r];
    for (int j = r + 1; j < k; ++j) s -= A[r * k + j] * (*g)[j];
    (*g)[r] = s / A[r * k + r];
  }
  return true;
}

int Scf::run(int nocc, int nbnd, double tol, int maxiter, double2* psi, double* eig_out, double* energies,
             int* iters_out, double* norm2_out) {
  Context& c = c_;
  const int nmix = std::max(1, std::min(kMaxMix, c.scf_nmix));
  int rc = alloc(nmix, nbnd);
  if (rc) return rc;
  ScfWork& w = *w_;
  SCK(cudaMemcpyAsync(w.vext, p_.vext.data(), sizeof(double) * nr_, cudaMemcpyHostToDevice, c.stream), "V_ext upload");
  HPSI_LAUNCH(c, HPSI_K_SCF, (k_norm_weight<<<grid_for(nr_), 256, 0, c.stream>>>(p_.n[0], p_.n[1], p_.n[2], rc_, omega_,
                                                                                 w.wgt)));
  std::vector<double> eig(nbnd), res(nbnd);
  int nhist = 0, head = 0;   // entries in the mixing history (oldest first) and the oldest's slot
  const size_t rb = sizeof(double) * nr_;
  for (int it = 0; it < maxiter; ++it) {
    // V[rho_in] into the context, then the lowest bands of H[V]
    double ehxc_in = 0.0;
    rc = hxc(w.rho_in, &ehxc_in);
    if (rc) return rc;
    double vsum = 0.0;
    rc = dot(w.vtot, nullptr, &vsum);
    if (rc) return rc;
    rc = set_potential(c, ik_, w.vtot, vsum / (double)nr_);
    if (rc) return rc;
    int dit = 0;
    rc = davidson_run(c, ik_, nbnd, c.scf_dav_tol, 1000, psi, eig.data(), &dit, res.data());
    if (rc && rc != HPSI_ENOTCONV) return rc;
    // rho_out and the scf norm of its difference from rho_in
    SCK(cudaMemsetAsync(w.rho_out, 0, rb, c.stream), "density clear");
    HPSI_LAUNCH(c, HPSI_K_SCF, (k_occ_weights<<<nocc, 256, 0, c.stream>>>(p_.npw, psi, 2.0 / omega_, w.occ)));
    rc = local_density(c, p_, psi, nocc, w.occ, w.rho_out);
    if (rc) return rc;
    double n2 = 0.0;
    rc = transform(w.rho_out, w.rho_in, &n2, false);   // box <- Fourier components of rho_out - rho_in
    if (rc) return rc;
    if (norm2_out) norm2_out[it] = n2;
    if (iters_out) *iters_out = it + 1;
    if (n2 < tol) {
      double band = 0.0;
      for (int i = 0; i < nocc; ++i) band += 2.0 * eig[i];
      double out_v = 0.0, in_v = 0.0, ehxc_out = 0.0;
      rc = dot(w.rho_out, w.vhxc, &out_v);
      if (!rc) rc = dot(w.rho_in, w.vhxc, &in_v);
      if (rc) return rc;
      const double dv = omega_ / (double)nr_;
      rc = hxc(w.rho_out, &ehxc_out);   // overwrites vhxc / vtot; the context keeps V[rho_in]
      if (rc) return rc;
      energies[0] = band - dv * out_v + ehxc_out;
      energies[1] = band - dv * in_v + ehxc_in;
      for (int i = 0; i < nbnd; ++i) eig_out[i] = eig[i];
      return HPSI_OK;
    }
    // mixing: append (rho_in, r = rho_out - rho_in, r(G)) to the history, a ring of nmix slots
    // (entry e, counted from the oldest kept, lives in slot (head + e) mod nmix)
    if (nhist == nmix) {
      head = (head + 1) % nmix;   // the oldest entry's slot is reused
      --nhist;
    }
    auto slot = [&](int e) { return (size_t)((head + e) % nmix) * nr_; };
    double* xn = w.xin + slot(nhist);
    double* rn = w.res + slot(nhist);
    double2* hn = w.rhat + slot(nhist);
    SCK(cudaMemcpyAsync(xn, w.rho_in, rb, cudaMemcpyDeviceToDevice, c.stream), "history");
    HPSI_LAUNCH(c, HPSI_K_SCF, (k_sub<<<grid_for(nr_), 256, 0, c.stream>>>(nr_, w.rho_out, w.rho_in, rn)));
    SCK(cudaMemcpyAsync(hn, w.box, 2 * rb, cudaMemcpyDeviceToDevice, c.stream), "history");
    ++nhist;
    // x = x_n - sum_j g_j (x_{j+1} - x_j), r = r_n - sum_j g_j (r_{j+1} - r_j), g minimising the
    // scf norm of r (least squares on the residual differences in the scf-norm metric)
    std::vector<double> g;
    int k = nhist - 1;
    while (k > 0) {
      std::vector<double> A((size_t)k * k), bv(k);
      // <dr_i, dr_j> = <h_{i+1} - h_i, h_{j+1} - h_j> expanded in the stored transforms h
      std::vector<double> H((size_t)(k + 1) * (k + 1));
      const int base = nhist - 1 - k;
      for (int i = 0; i <= k; ++i)
        for (int j = i; j <= k; ++j) {
          double v = 0.0;
          rc = wdot(w.rhat + slot(base + i), w.rhat + slot(base + j), &v);
          if (rc) return rc;
          H[(size_t)i * (k + 1) + j] = H[(size_t)j * (k + 1) + i] = v;
        }
      auto h = [&](int i, int j) { return H[(size_t)i * (k + 1) + j]; };
      for (int i = 0; i < k; ++i) {
        for (int j = 0; j < k; ++j) A[(size_t)i * k + j] = h(i + 1, j + 1) - h(i + 1, j) - h(i, j + 1) + h(i, j);
        bv[i] = h(i + 1, k) - h(i, k);
      }
      if (small_solve(k, A, bv, &g)) break;
      --k;   // drop the oldest pair from the combination
      g.clear();
    }
    SCK(cudaMemcpyAsync(w.rho_in, xn, rb, cudaMemcpyDeviceToDevice, c.stream), "mix");
    SCK(cudaMemcpyAsync(w.tmp, rn, rb, cudaMemcpyDeviceToDevice, c.stream), "mix");
    const int base = nhist - 1 - k;
    for (int j = 0; j < (int)g.size(); ++j) {
      const double* x0 = w.xin + slot(base + j);
      const double* x1 = w.xin + slot(base + j + 1);
      const double* r0 = w.res + slot(base + j);
      const double* r1 = w.res + slot(base + j + 1);
      HPSI_LAUNCH(c, HPSI_K_SCF, (k_axpby<<<grid_for(nr_), 256, 0, c.stream>>>(nr_, -g[j], x1, 1.0, w.rho_in)));
      HPSI_LAUNCH(c, HPSI_K_SCF, (k_axpby<<<grid_for(nr_), 256, 0, c.stream>>>(nr_, g[j], x0, 1.0, w.rho_in)));
      HPSI_LAUNCH(c, HPSI_K_SCF, (k_axpby<<<grid_for(nr_), 256, 0, c.stream>>>(nr_, -g[j], r1, 1.0, w.tmp)));
      HPSI_LAUNCH(c, HPSI_K_SCF, (k_axpby<<<grid_for(nr_), 256, 0, c.stream>>>(nr_, g[j], r0, 1.0, w.tmp)));
    }
    HPSI_LAUNCH(c, HPSI_K_SCF, (k_axpby<<<grid_for(nr_), 256, 0, c.stream>>>(nr_, c.scf_beta, w.tmp, 1.0, w.rho_in)));
    SCK(cudaGetLastError(), "mixing kernels");
  }
  for (int i = 0; i < nbnd; ++i) eig_out[i] = eig[i];
  return fail(c, HPSI_ENOTCONV, "hpsi_scf: not self-consistent within maxiter");
}

}  // namespace

}  // namespace hpsi

using namespace hpsi;

extern "C" int hpsi_scf(hpsi_ctx* ctx, int ik, int nocc, int nbnd, double tol, int maxiter, void* psi_inout,
                        double* rho_inout, double* eig_out, double* energies_out, int* iters_out, double* norm2_out) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  if (ik < 0 || ik >= (int)c.probs.size()) return fail(c, HPSI_EINVAL, "hpsi_scf: problem index out of range");
  const Problem& p = c.probs[ik];
  if (nocc < 1 || nbnd < nocc || (long long)nbnd * basis_of(c) > p.npw)
    return fail(c, HPSI_EINVAL, "hpsi_scf: need 1 <= nocc <= nbnd and nbnd times the basis factor <= npw");
  if (!(tol > 0.0) || maxiter < 1 || !psi_inout || !rho_inout || !eig_out || !energies_out)
    return fail(c, HPSI_EINVAL, "hpsi_scf: bad argument");
  if (c.precision != HPSI_FP64) return fail(c, HPSI_EINVAL, "hpsi_scf: needs a float64 context");
  const int kind = pointer_kind(psi_inout);
  if (kind < 0) return fail(c, HPSI_EINVAL, "hpsi_scf: psi_inout is not a valid pointer");
  const size_t pb = sizeof(double2) * (size_t)nbnd * p.npw;
  double2* dpsi = static_cast<double2*>(psi_inout);
  if (kind == 0) {
    int rc = ensure_buffer(c, &c.ws.stage_in, &c.ws.stage_in_bytes, pb);
    if (rc) return rc;
    dpsi = static_cast<double2*>(c.ws.stage_in);
    cudaError_t e = cudaMemcpyAsync(dpsi, psi_inout, pb, cudaMemcpyHostToDevice, c.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "hpsi_scf host->device copy");
  }
  Scf s(c, ik);
  int rc = s.alloc(std::max(1, std::min(kMaxMix, c.scf_nmix)), nbnd);
  if (rc) return rc;
  const int n1 = p.n[0], n2 = p.n[1], n3 = p.n[2];
  const size_t nr = (size_t)n1 * n2 * n3;
  std::vector<double> t(nr);
  for (int j1 = 0; j1 < n1; ++j1)
    for (int j2 = 0; j2 < n2; ++j2)
      for (int j3 = 0; j3 < n3; ++j3) t[((size_t)j3 * n2 + j2) * n1 + j1] = rho_inout[((size_t)j1 * n2 + j2) * n3 + j3];
  cudaError_t e = cudaMemcpyAsync(s.w_->rho_in, t.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "hpsi_scf density upload");
  rc = s.run(nocc, nbnd, tol, maxiter, dpsi, eig_out, energies_out, iters_out, norm2_out);
  if (rc != HPSI_OK && rc != HPSI_ENOTCONV) return rc;
  e = cudaMemcpyAsync(t.data(), s.w_->rho_in, sizeof(double) * nr, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess && kind == 0) e = cudaMemcpyAsync(psi_inout, dpsi, pb, cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "hpsi_scf result copy");
  for (int j1 = 0; j1 < n1; ++j1)
    for (int j2 = 0; j2 < n2; ++j2)
      for (int j3 = 0; j3 < n3; ++j3) rho_inout[((size_t)j1 * n2 + j2) * n3 + j3] = t[((size_t)j3 * n2 + j2) * n1 + j1];
  const int rc2 = check_device_error(c);
  return rc2 ? rc2 : rc;
}
