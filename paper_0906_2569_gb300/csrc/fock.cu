// Fock exchange at the Gamma point (paper App. A.5), on the GPU.
//
// For closed shells with physical orbitals phi = psi / Omega^(1/2) (psi(r) = sum_G psi(G) e^{iG.r},
// sum_G |psi(G)|^2 = 1):
//   (V_x psi_b)(r) = - sum_j psi_j(r) v_bj(r),  v_bj = Coulomb potential of n_bj = conj(psi_j) psi_b / Omega,
//   v(G) = 4 pi n(G) / G^2 for G != 0 and 4 pi n(0) x_div at G = 0,
// with the Gygi-Baldereschi constant of the single q point and auxiliary function e^{-alpha G^2}/G^2,
//   x_div = Omega / (2 pi)^3 * 2 pi^(3/2) / alpha^(1/2) - sum_{G != 0 in the box} e^{-alpha G^2} / G^2.
// The result is returned on the G-sphere: (V_x psi)(G) = N_r^-1 sum_j e^{-iG.r_j} (V_x psi)(r_j).
// With one q point the paper's estimate of the 0/0 term from a coarser grid is not available; that
// term is left out.
//
// Steps per band b (all occupied j at once, as a batch of boxes): the occupied orbitals are in real
// space once; psi_b is scattered into a box and transformed; the codensities of every j are formed,
// transformed forward, multiplied by the Coulomb kernel, transformed back, multiplied by psi_j and
// summed over j into the band's output box, which is transformed forward and gathered on the sphere.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "box_fft.cuh"
#include "hpsi_internal.h"

namespace hpsi {

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kRed = 304;

struct Recip {
  double b[9];
};

__device__ __forceinline__ int sfreq(int j, int n) { return 2 * j < n ? j : j - n; }

__device__ __forceinline__ double bsum(double s) {
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

// Coulomb kernel 4 pi / G^2 (entry G = 0 set later from x_div), scaled by scale; partial sums of
// e^{-alpha G^2} / G^2 over G != 0 for x_div.
__global__ void __launch_bounds__(256) k_coulomb(int n1, int n2, int n3, Recip rc, double alpha, double scale,
                                                 double* __restrict__ kern, double* __restrict__ partial) {
  const size_t n = (size_t)n1 * n2 * n3;
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int j1 = (int)(i % n1), j2 = (int)((i / n1) % n2), j3 = (int)(i / ((size_t)n1 * n2));
    const double m1 = sfreq(j1, n1), m2 = sfreq(j2, n2), m3 = sfreq(j3, n3);
    const double gx = m1 * rc.b[0] + m2 * rc.b[3] + m3 * rc.b[6];
    const double gy = m1 * rc.b[1] + m2 * rc.b[4] + m3 * rc.b[7];
    const double gz = m1 * rc.b[2] + m2 * rc.b[5] + m3 * rc.b[8];
    const double g2 = gx * gx + gy * gy + gz * gz;
    if (g2 > 1e-12) {
      kern[i] = scale * 4.0 * kPi / g2;
      acc += exp(-alpha * g2) / g2;
    } else {
      kern[i] = 0.0;
    }
  }
  acc = bsum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

// psi [nb][npw] on the sphere -> boxes [nb][n3][n2][n1] (zero elsewhere); box index of G from its
// Miller indices.  One thread per (G, band).
__global__ void k_sphere_to_box(int npw, int nb, const int* __restrict__ boxidx, const double2* __restrict__ psi,
                                double2* __restrict__ boxes, size_t nr) {
  const int b = blockIdx.y;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x)
    boxes[(size_t)b * nr + boxidx[g]] = psi[(size_t)b * npw + g];
}

// out [nb][npw] = scale * boxes at the sphere's points (accumulate: out += ...)
__global__ void k_box_to_sphere(int npw, int nb, const int* __restrict__ boxidx, const double2* __restrict__ boxes,
                                size_t nr, double scale, int accumulate, double2* __restrict__ out) {
  const int b = blockIdx.y;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npw; g += gridDim.x * blockDim.x) {
    const double2 v = boxes[(size_t)b * nr + boxidx[g]];
    double2* o = out + (size_t)b * npw + g;
    if (accumulate) *o = make_double2(o->x + scale * v.x, o->y + scale * v.y);
    else *o = make_double2(scale * v.x, scale * v.y);
  }
}

// codensities n_j(r) = conj(phi_j(r)) psi(r) * scale for every occupied j (box j of co)
__global__ void k_codensity(size_t nr, int nocc, const double2* __restrict__ occ_r, const double2* __restrict__ psi_r,
                            double scale, double2* __restrict__ co) {
  const int j = blockIdx.y;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += (size_t)gridDim.x * blockDim.x) {
    const double2 a = occ_r[(size_t)j * nr + i], b = psi_r[i];
    co[(size_t)j * nr + i] = make_double2(scale * (a.x * b.x + a.y * b.y), scale * (a.x * b.y - a.y * b.x));
  }
}

// co_j(G) *= kern(G) (kern holds 4 pi / G^2 / N_r, and 4 pi x_div / N_r at G = 0)
__global__ void k_apply_kernel(size_t nr, int nocc, const double* __restrict__ kern, double2* __restrict__ co) {
  const int j = blockIdx.y;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += (size_t)gridDim.x * blockDim.x) {
    const double k = kern[i];
    double2* v = co + (size_t)j * nr + i;
    *v = make_double2(k * v->x, k * v->y);
  }
}

// out(r) = - sum_j phi_j(r) v_j(r)
__global__ void k_exchange_sum(size_t nr, int nocc, const double2* __restrict__ occ_r, const double2* __restrict__ v,
                               double2* __restrict__ out) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += (size_t)gridDim.x * blockDim.x) {
    double sx = 0.0, sy = 0.0;
    for (int j = 0; j < nocc; ++j) {
      const double2 a = occ_r[(size_t)j * nr + i], b = v[(size_t)j * nr + i];
      sx += a.x * b.x - a.y * b.y;
      sy += a.x * b.y + a.y * b.x;
    }
    out[i] = make_double2(-sx, -sy);
  }
}

// partial[block] = Re sum conj(a) b over n complex elements
__global__ void __launch_bounds__(256) k_cdot(size_t n, const double2* __restrict__ a, const double2* __restrict__ b,
                                              double* __restrict__ partial) {
  double acc = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc += a[i].x * b[i].x + a[i].y * b[i].y;
  acc = bsum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

int grid_n(size_t n) { return (int)std::min<size_t>(4096, (n + 255) / 256); }

}  // namespace

struct FockWork {
  size_t nr = 0;
  int nocc = 0;
  double2* occ_r = nullptr;   // [nocc][nr]
  double2* co = nullptr;      // [nocc][nr]
  double2* psi_r = nullptr;   // [nr]
  double2* out_r = nullptr;   // [nr]
  double* kern = nullptr;     // [nr]
  int* boxidx = nullptr;      // [npw]
  int npw = 0;
  double* partial = nullptr;  // [kRed]
};

static void free_fock(FockWork& w) {
  for (double2* p : {w.occ_r, w.co, w.psi_r, w.out_r}) cudaFree(p);
  cudaFree(w.kern);
  cudaFree(w.boxidx);
  cudaFree(w.partial);
  w = FockWork();
}

void fock_release(Context& c) {
  FockWork* w = reinterpret_cast<FockWork*>(c.fock);
  if (!w) return;
  free_fock(*w);
  delete w;
  c.fock = nullptr;
}

#define FCK(x, what)                                      \
  do {                                                    \
    cudaError_t e_ = (x);                                 \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

static int fock_alloc(Context& c, const Problem& p, int nocc, FockWork** out) {
  FockWork* w = reinterpret_cast<FockWork*>(c.fock);
  if (!w) {
    w = new FockWork();
    c.fock = w;
  }
  *out = w;
  const size_t nr = (size_t)p.n[0] * p.n[1] * p.n[2];
  if (w->nr == nr && w->nocc >= nocc && w->npw == p.npw) return HPSI_OK;
  free_fock(*w);
  auto al = [&](void** q, size_t bytes) -> bool {
    if (cudaMalloc(q, std::max<size_t>(bytes, 256)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  const size_t cb = sizeof(double2) * nr;
  const bool ok = al((void**)&w->occ_r, cb * nocc) && al((void**)&w->co, cb * nocc) && al((void**)&w->psi_r, cb) &&
                  al((void**)&w->out_r, cb) && al((void**)&w->kern, sizeof(double) * nr) &&
                  al((void**)&w->boxidx, sizeof(int) * p.npw) && al((void**)&w->partial, sizeof(double) * kRed);
  if (!ok) {
    free_fock(*w);
    return fail(c, HPSI_ENOMEM, "hpsi_fock_apply: device allocation failed");
  }
  w->nr = nr;
  w->nocc = nocc;
  w->npw = p.npw;
  // box position of every G of the sphere: (m_i mod n_i), x fastest
  std::vector<int> idx(p.npw);
  for (int g = 0; g < p.npw; ++g) {
    int j[3];
    for (int a = 0; a < 3; ++a) {
      const int m = p.miller[(size_t)g * 3 + a];
      j[a] = ((m % p.n[a]) + p.n[a]) % p.n[a];
    }
    idx[g] = (j[2] * p.n[1] + j[1]) * p.n[0] + j[0];
  }
  FCK(cudaMemcpyAsync(w->boxidx, idx.data(), sizeof(int) * p.npw, cudaMemcpyHostToDevice, c.stream), "box map");
  FCK(cudaStreamSynchronize(c.stream), "box map");
  return HPSI_OK;
}

static int fock_run(Context& c, int ik, int nocc, const double2* occ, const double2* psi, double2* vx, int nbnd,
                    double alpha, double* ex_out) {
  const Problem& p = c.probs[ik];
  FockWork* w = nullptr;
  int rc = fock_alloc(c, p, nocc, &w);
  if (rc) return rc;
  const size_t nr = w->nr;
  const double omega = std::fabs(p.cell[0] * (p.cell[4] * p.cell[8] - p.cell[5] * p.cell[7]) -
                                 p.cell[1] * (p.cell[3] * p.cell[8] - p.cell[5] * p.cell[6]) +
                                 p.cell[2] * (p.cell[3] * p.cell[7] - p.cell[4] * p.cell[6]));
  Recip r;
  for (int i = 0; i < 9; ++i) r.b[i] = p.recip[i];
  // Coulomb kernel with the 1/N_r of the forward transform folded in, and x_div
  HPSI_LAUNCH(c, HPSI_K_FOCK, (k_coulomb<<<kRed, 256, 0, c.stream>>>(p.n[0], p.n[1], p.n[2], r, alpha, 1.0 / (double)nr,
                                                                     w->kern, w->partial)));
  std::vector<double> part(kRed);
  FCK(cudaMemcpyAsync(part.data(), w->partial, sizeof(double) * kRed, cudaMemcpyDeviceToHost, c.stream), "x_div sum");
  FCK(cudaStreamSynchronize(c.stream), "x_div sum");
  double s = 0.0;
  for (double v : part) s += v;
  const double xdiv = omega / std::pow(2.0 * kPi, 3) * 2.0 * std::pow(kPi, 1.5) / std::sqrt(alpha) - s;
  const double k0 = 4.0 * kPi * xdiv / (double)nr;
  FCK(cudaMemcpyAsync(w->kern, &k0, sizeof(double), cudaMemcpyHostToDevice, c.stream), "G = 0 kernel");
  // occupied orbitals in real space
  FCK(cudaMemsetAsync(w->occ_r, 0, sizeof(double2) * nr * nocc, c.stream), "clear");
  HPSI_LAUNCH(c, HPSI_K_FOCK, (k_sphere_to_box<<<dim3(grid_n(p.npw), nocc), 256, 0, c.stream>>>(p.npw, nocc, w->boxidx,
                                                                                                 occ, w->occ_r, nr)));
  rc = box_fft(c, p, w->occ_r, nocc, +1, HPSI_K_FOCK);
  if (rc) return rc;
  const double inv_omega = 1.0 / omega;
  for (int b = 0; b < nbnd; ++b) {
    FCK(cudaMemsetAsync(w->psi_r, 0, sizeof(double2) * nr, c.stream), "clear");
    HPSI_LAUNCH(c, HPSI_K_FOCK, (k_sphere_to_box<<<dim3(grid_n(p.npw), 1), 256, 0, c.stream>>>(
                                    p.npw, 1, w->boxidx, psi + (size_t)b * p.npw, w->psi_r, nr)));
    rc = box_fft(c, p, w->psi_r, 1, +1, HPSI_K_FOCK);
    if (rc) return rc;
    HPSI_LAUNCH(c, HPSI_K_FOCK, (k_codensity<<<dim3(grid_n(nr), nocc), 256, 0, c.stream>>>(nr, nocc, w->occ_r, w->psi_r,
                                                                                            inv_omega, w->co)));
    rc = box_fft(c, p, w->co, nocc, -1, HPSI_K_FOCK);
    if (rc) return rc;
    HPSI_LAUNCH(c, HPSI_K_FOCK, (k_apply_kernel<<<dim3(grid_n(nr), nocc), 256, 0, c.stream>>>(nr, nocc, w->kern, w->co)));
    rc = box_fft(c, p, w->co, nocc, +1, HPSI_K_FOCK);
    if (rc) return rc;
    HPSI_LAUNCH(c, HPSI_K_FOCK, (k_exchange_sum<<<grid_n(nr), 256, 0, c.stream>>>(nr, nocc, w->occ_r, w->co, w->out_r)));
    rc = box_fft(c, p, w->out_r, 1, -1, HPSI_K_FOCK);
    if (rc) return rc;
    HPSI_LAUNCH(c, HPSI_K_FOCK, (k_box_to_sphere<<<dim3(grid_n(p.npw), 1), 256, 0, c.stream>>>(
                                    p.npw, 1, w->boxidx, w->out_r, nr, 1.0 / (double)nr, 0, vx + (size_t)b * p.npw)));
  }
  FCK(cudaGetLastError(), "exchange kernels");
  if (ex_out) {
    HPSI_LAUNCH(c, HPSI_K_FOCK, (k_cdot<<<kRed, 256, 0, c.stream>>>((size_t)nbnd * p.npw, psi, vx, w->partial)));
    FCK(cudaMemcpyAsync(part.data(), w->partial, sizeof(double) * kRed, cudaMemcpyDeviceToHost, c.stream), "E_x");
    FCK(cudaStreamSynchronize(c.stream), "E_x");
    double ex = 0.0;
    for (double v : part) ex += v;
    *ex_out = ex;
  }
  return HPSI_OK;
}

}  // namespace hpsi

using namespace hpsi;

extern "C" int hpsi_fock_apply(hpsi_ctx* ctx, int ik, int nocc, const void* occ, const void* psi_in, void* vx_out,
                               int nbnd, double alpha, double* ex_out) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  if (ik < 0 || ik >= (int)c.probs.size()) return fail(c, HPSI_EINVAL, "hpsi_fock_apply: problem index out of range");
  const Problem& p = c.probs[ik];
  if (p.k[0] != 0.0 || p.k[1] != 0.0 || p.k[2] != 0.0)
    return fail(c, HPSI_EINVAL, "hpsi_fock_apply: the exchange operator is implemented at k = q = 0 only");
  if (nocc < 1 || nbnd < 0 || !(alpha > 0.0) || !occ || (nbnd > 0 && (!psi_in || !vx_out)))
    return fail(c, HPSI_EINVAL, "hpsi_fock_apply: bad argument");
  if (nbnd == 0) return HPSI_OK;
  if (pointer_kind(occ) != 1 || pointer_kind(psi_in) != 1 || pointer_kind(vx_out) != 1)
    return fail(c, HPSI_EINVAL, "hpsi_fock_apply: occ, psi_in and vx_out must be device memory");
  const size_t bytes = sizeof(double2) * (size_t)nbnd * p.npw;
  const char* a0 = static_cast<const char*>(psi_in);
  const char* b0 = static_cast<const char*>(vx_out);
  const char* o0 = static_cast<const char*>(occ);
  const size_t ob = sizeof(double2) * (size_t)nocc * p.npw;
  if ((a0 < b0 + bytes && b0 < a0 + bytes) || (o0 < b0 + bytes && b0 < o0 + ob))
    return fail(c, HPSI_EINVAL, "hpsi_fock_apply: vx_out overlaps an input");
  int rc = fock_run(c, ik, nocc, static_cast<const double2*>(occ), static_cast<const double2*>(psi_in),
                    static_cast<double2*>(vx_out), nbnd, alpha, ex_out);
  if (rc) return rc;
  return ex_out ? check_device_error(c) : HPSI_OK;
}
