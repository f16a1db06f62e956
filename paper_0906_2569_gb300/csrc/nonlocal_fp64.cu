// Separable nonlocal term in float64 (paper Sec. 3: Kleinman-Bylander separable NC projectors):
//   becp[b][p] = <beta_p|psi_b> = sum_G conj(beta_p(G)) psi_b(G)            (calbec)
//   w[b][p]    = sum_q D_pq becp[b][q]                                          (D-scale, CSR of D)
//   hpsi_b(G) += sum_p beta_p(G) w[b][p]                                        (add_vuspsi)
// On GB300 float64 runs at ~1.2 TFLOP/s on the CUDA cores (the FP64 MMA path is not faster), so
// these are plain shared-memory-tiled complex GEMMs whose inner loop is DFMA-bound; calbec
// (P x nb outputs, K = npw) splits K across CTAs and reduces the partials deterministically in
// the D-scale kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "hpsi_internal.h"

namespace hpsi {

namespace {

#include "nonlocal_tiles.cuh"

__global__ void __launch_bounds__(256) k_calbec64(int npw, int nproj, int nb, int kchunk,
                                                  const double2* __restrict__ beta,
                                                  const double2* __restrict__ psi, double2* __restrict__ part) {
  __shared__ double2 sm[CB_SMEM];
  calbec_tile(npw, nproj, nb, kchunk, beta, psi, part, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

__global__ void k_dscale64(int nproj, int nb, int nsplit, const double2* __restrict__ part,
                           const int* __restrict__ rowptr, const int* __restrict__ col,
                           const double2* __restrict__ val, double2* __restrict__ w) {
  dscale_one(blockIdx.x * blockDim.x + threadIdx.x, nproj, nb, nsplit, part, rowptr, col, val, w);
}

__global__ void __launch_bounds__(256) k_addvus64(int npw, int nproj, int nb, const double2* __restrict__ w,
                                                  const double2* __restrict__ beta, double2* __restrict__ hpsi) {
  __shared__ double2 sm[AV_SMEM];
  addvus_tile(npw, nproj, nb, w, beta, hpsi, blockIdx.x, blockIdx.y, sm);
}

__global__ void __launch_bounds__(256) k_calbec64_batch(const __grid_constant__ NlBatch bt) {
  const int i = find_item(bt.off_cal, bt.nitems, blockIdx.x);
  const NlItem& a = bt.item[i];
  const int l = blockIdx.x - bt.off_cal[i];
  const int tp = l % a.tilesp, r = l / a.tilesp;
  __shared__ double2 sm[CB_SMEM];
  if (a.tp == 8)
    calbec_tile_t<8>(a.npw, a.nproj, a.nb, a.kchunk, a.beta, a.psi, a.part, tp, r % a.tilesb, r / a.tilesb, sm);
  else if (a.tp == 16)
    calbec_tile_t<16>(a.npw, a.nproj, a.nb, a.kchunk, a.beta, a.psi, a.part, tp, r % a.tilesb, r / a.tilesb, sm);
  else
    calbec_tile_t<CB_TP>(a.npw, a.nproj, a.nb, a.kchunk, a.beta, a.psi, a.part, tp, r % a.tilesb, r / a.tilesb, sm);
}

__global__ void __launch_bounds__(256) k_dscale64_batch(const __grid_constant__ NlBatch bt) {
  const int i = find_item(bt.off_ds, bt.nitems, blockIdx.x);
  const NlItem& a = bt.item[i];
  dscale_one((blockIdx.x - bt.off_ds[i]) * blockDim.x + threadIdx.x, a.nproj, a.nb, a.nsplit, a.part, a.rowptr,
             a.col, a.dval, a.w);
}

__global__ void __launch_bounds__(256) k_addvus64_batch(const __grid_constant__ NlBatch bt) {
  const int i = find_item(bt.off_add, bt.nitems, blockIdx.x);
  const NlItem& a = bt.item[i];
  const int l = blockIdx.x - bt.off_add[i];
  __shared__ double2 sm[AV_SMEM];
  addvus_tile(a.npw, a.nproj, a.nb, a.w, a.beta, a.hpsi, l % a.gtiles, l / a.gtiles, sm);
}

// ---- Gamma-point real form (Sec. 4) ----
// Real orbitals in real-basis coordinates x (nr = 2 nh reals: (c(0), 0) at G = 0, sqrt2 (Re c, Im c)
// elsewhere) and projectors rephased so that beta'(-G) = conj(beta'(G)), in the same coordinates
// (betar): <beta'_p|psi> = betar_p . x, D' is real, and V_NL psi has the coordinates
// sum_p betar_p (D' becp)_p.  Three real GEMMs, half the float64 work of the packed complex form.

constexpr double kSqrt2r = 1.4142135623730950488;
constexpr int RB_TP = 32;   // projectors per CTA
constexpr int RB_TB = 32;   // bands per CTA
constexpr int RB_TK = 64;   // coordinates per shared-memory tile

// part[split][b][p] = sum_{r in split} betar[p][r] x[b][r]; scaled = 0: x holds coefficients and
// r >= 2 is multiplied by sqrt2 on load
template <typename R>
__global__ void __launch_bounds__(256) k_calbec64r(int nr, int nproj, int nb, int kchunk, int scaled,
                                                   const double* __restrict__ betar, const R* __restrict__ x,
                                                   double* __restrict__ part) {
  __shared__ double sb[RB_TP][RB_TK + 1];
  __shared__ double sx[RB_TB][RB_TK + 1];
  const int p0 = blockIdx.x * RB_TP, b0 = blockIdx.y * RB_TB, split = blockIdx.z;
  const int rbeg = split * kchunk, rend = min(nr, rbeg + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // tx -> p, ty -> b
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int r0 = rbeg; r0 < rend; r0 += RB_TK) {
    for (int i = threadIdx.x; i < RB_TP * RB_TK; i += 256) {
      const int row = i / RB_TK, cc = i % RB_TK, r = r0 + cc;
      const bool in = r < rend;
      sb[row][cc] = (p0 + row < nproj && in) ? betar[(size_t)(p0 + row) * nr + r] : 0.0;
      double v = (b0 + row < nb && in) ? (double)x[(size_t)(b0 + row) * nr + r] : 0.0;
      if (!scaled && r >= 2) v *= kSqrt2r;
      sx[row][cc] = v;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < RB_TK; ++kk) {
      const double a0 = sb[tx][kk], a1 = sb[tx + 16][kk];
      const double y0 = sx[ty][kk], y1 = sx[ty + 16][kk];
      acc[0][0] = fma(a0, y0, acc[0][0]);
      acc[0][1] = fma(a0, y1, acc[0][1]);
      acc[1][0] = fma(a1, y0, acc[1][0]);
      acc[1][1] = fma(a1, y1, acc[1][1]);
    }
    __syncthreads();
  }
  double* out = part + (size_t)split * nb * nproj;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int pp = p0 + tx + 16 * i, b = b0 + ty + 16 * j;
      if (pp < nproj && b < nb) out[(size_t)b * nproj + pp] = acc[i][j];
    }
}

// w[b][p] = sum_{q in row p of D} D'_pq sum_s part[s][b][q]
__global__ void k_dscale64r(int nproj, int nb, int nsplit, const double* __restrict__ part,
                            const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, double* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nproj * nb) return;
  const int b = i / nproj, p = i % nproj;
  double acc = 0.0;
  for (int e = rowptr[p]; e < rowptr[p + 1]; ++e) {
    const int q = col[e];
    double s = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) s += part[((size_t)sp * nb + b) * nproj + q];
    acc = fma(val[e], s, acc);
  }
  w[i] = acc;
}

constexpr int RA_TR = 64;   // coordinates per CTA
constexpr int RA_TB = 32;   // bands per CTA
constexpr int RA_TP = 32;   // projectors per shared-memory tile

// out[b][r] = sum_p w[b][p] betar[p][r]
__global__ void __launch_bounds__(256) k_addvus64r(int nr, int nproj, int nb, const double* __restrict__ w,
                                                   const double* __restrict__ betar, double* __restrict__ out) {
  __shared__ double sb[RA_TP][RA_TR];
  __shared__ double sw[RA_TB][RA_TP + 1];
  const int r0 = blockIdx.x * RA_TR, b0 = blockIdx.y * RA_TB;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;   // tx -> r, ty -> bands ty + 4 j
  double acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0;
  for (int q0 = 0; q0 < nproj; q0 += RA_TP) {
    for (int i = threadIdx.x; i < RA_TP * RA_TR; i += 256) {
      const int row = i / RA_TR, cc = i % RA_TR;
      const int q = q0 + row, r = r0 + cc;
      sb[row][cc] = (q < nproj && r < nr) ? betar[(size_t)q * nr + r] : 0.0;
    }
    for (int i = threadIdx.x; i < RA_TB * RA_TP; i += 256) {
      const int row = i / RA_TP, cc = i % RA_TP;
      const int b = b0 + row, q = q0 + cc;
      sw[row][cc] = (b < nb && q < nproj) ? w[(size_t)b * nproj + q] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < RA_TP; ++kk) {
      const double xv = sb[kk][tx];
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[j] = fma(sw[ty + 4 * j][kk], xv, acc[j]);
    }
    __syncthreads();
  }
  const int r = r0 + tx;
  if (r < nr) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int b = b0 + ty + 4 * j;
      if (b < nb) out[(size_t)b * nr + r] = acc[j];
    }
  }
}

// ---- double-float calbec (the projections of the mixed solve's final quotients) ----
// Pairs of floats (hi + lo, ~48 bits) multiplied and accumulated with error-free transformations
// on the float32 pipes (Knuth's TwoSum, Dekker's FastTwoSum, the FMA split of a product); the _rn
// intrinsics keep the compiler from contracting or reassociating them.
__device__ __forceinline__ float2 dfr_fast(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 dfr_mac(float2 acc, float2 a, float2 u) {
  const float p = __fmul_rn(a.x, u.x);
  float e = __fmaf_rn(a.x, u.x, -p);
  e = __fmaf_rn(a.x, u.y, e);
  e = __fmaf_rn(a.y, u.x, e);
  const float s = __fadd_rn(acc.x, p);
  const float bb = __fsub_rn(s, acc.x);
  const float err = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  return dfr_fast(s, __fadd_rn(err, __fadd_rn(acc.y, e)));
}
__device__ __forceinline__ float2 dfr_of(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

// out[i] = pairs of in[i] (x sqrt2 for coordinates r >= 2 of each nr-long row when !scaled)
template <typename R>
__global__ void k_to_df(size_t n, int nr, int scaled, const R* __restrict__ in, float2* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double v = (double)in[i];
    if (!scaled && (int)(i % nr) >= 2) v *= kSqrt2r;
    out[i] = dfr_of(v);
  }
}

// part[split][b][p] = sum_{r in split} betar[p][r] x[b][r] in pairs, written as float64
__global__ void __launch_bounds__(256) k_calbec_df(int nr, int nproj, int nb, int kchunk,
                                                   const float2* __restrict__ betar, const float2* __restrict__ x,
                                                   double* __restrict__ part) {
  __shared__ float2 sb[RB_TP][RB_TK + 1];
  __shared__ float2 sx[RB_TB][RB_TK + 1];
  const int p0 = blockIdx.x * RB_TP, b0 = blockIdx.y * RB_TB, split = blockIdx.z;
  const int rbeg = split * kchunk, rend = min(nr, rbeg + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // tx -> p, ty -> b
  const float2 z = make_float2(0.f, 0.f);
  float2 c00 = z, c01 = z, c10 = z, c11 = z;
  for (int r0 = rbeg; r0 < rend; r0 += RB_TK) {
    for (int i = threadIdx.x; i < RB_TP * RB_TK; i += 256) {
      const int row = i / RB_TK, cc = i % RB_TK, r = r0 + cc;
      const bool in = r < rend;
      sb[row][cc] = (p0 + row < nproj && in) ? betar[(size_t)(p0 + row) * nr + r] : z;
      sx[row][cc] = (b0 + row < nb && in) ? x[(size_t)(b0 + row) * nr + r] : z;
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < RB_TK; ++kk) {
      const float2 a0 = sb[tx][kk], a1 = sb[tx + 16][kk];
      const float2 y0 = sx[ty][kk], y1 = sx[ty + 16][kk];
      c00 = dfr_mac(c00, a0, y0);
      c01 = dfr_mac(c01, a0, y1);
      c10 = dfr_mac(c10, a1, y0);
      c11 = dfr_mac(c11, a1, y1);
    }
    __syncthreads();
  }
  double* out = part + (size_t)split * nb * nproj;
  const int pa = p0 + tx, pb = pa + 16, ba = b0 + ty, bb = ba + 16;
  if (pa < nproj && ba < nb) out[(size_t)ba * nproj + pa] = (double)c00.x + (double)c00.y;
  if (pa < nproj && bb < nb) out[(size_t)bb * nproj + pa] = (double)c01.x + (double)c01.y;
  if (pb < nproj && ba < nb) out[(size_t)ba * nproj + pb] = (double)c10.x + (double)c10.y;
  if (pb < nproj && bb < nb) out[(size_t)bb * nproj + pb] = (double)c11.x + (double)c11.y;
}

}  // namespace

int gamma_prepare_df(Context& c, Problem& p) {
  if (p.nproj == 0 || p.d_betar_df) return HPSI_OK;
  const int nr = 2 * ((p.npw + 1) / 2);
  const size_t n = (size_t)p.nproj * nr;
  if (cudaMalloc((void**)&p.d_betar_df, sizeof(float2) * n) != cudaSuccess) {
    cudaGetLastError();
    p.d_betar_df = nullptr;
    return fail(c, HPSI_ENOMEM, "device allocation of the Gamma-form double-float projectors failed");
  }
  HPSI_LAUNCH(c, HPSI_K_GAMMA, (k_to_df<double><<<4 * c.sm_count, 256, 0, c.stream>>>(n, nr, 1, p.d_betar,
                                                                                      p.d_betar_df)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "Gamma-form double-float projector setup");
  return HPSI_OK;
}

int gamma_w_df(Context& c, const Problem& p, const void* x, bool x32, int nb, bool scaled, double** wout) {
  if (!p.d_betar_df) return fail(c, HPSI_EINVAL, "Gamma-form double-float projectors are not prepared");
  const int nr = 2 * ((p.npw + 1) / 2);
  const size_t nx = (size_t)nb * nr;
  int rc = ensure_buffer(c, &c.ws.gdf, &c.ws.gdfbytes, sizeof(float2) * nx);
  if (rc) return rc;
  float2* xdf = static_cast<float2*>(c.ws.gdf);
  if (x32)
    HPSI_LAUNCH(c, HPSI_K_CALBEC, (k_to_df<float><<<4 * c.sm_count, 256, 0, c.stream>>>(
                                      nx, nr, scaled ? 1 : 0, static_cast<const float*>(x), xdf)));
  else
    HPSI_LAUNCH(c, HPSI_K_CALBEC, (k_to_df<double><<<4 * c.sm_count, 256, 0, c.stream>>>(
                                      nx, nr, scaled ? 1 : 0, static_cast<const double*>(x), xdf)));
  const int tilesp = (p.nproj + RB_TP - 1) / RB_TP, tilesb = (nb + RB_TB - 1) / RB_TB;
  int nsplit = std::max(1, (3 * c.sm_count) / std::max(1, tilesp * tilesb));
  int kchunk = (nr + nsplit - 1) / nsplit;
  kchunk = std::max(RB_TK * 2, ((kchunk + RB_TK - 1) / RB_TK) * RB_TK);
  nsplit = (nr + kchunk - 1) / kchunk;
  rc = ensure_buffer(c, &c.ws.part, &c.ws.partbytes, sizeof(double) * (size_t)nsplit * nb * p.nproj);
  if (rc) return rc;
  rc = ensure_buffer(c, &c.ws.w, &c.ws.wbytes, sizeof(double) * (size_t)nb * p.nproj);
  if (rc) return rc;
  double* part = static_cast<double*>(c.ws.part);
  double* w = static_cast<double*>(c.ws.w);
  HPSI_LAUNCH(c, HPSI_K_CALBEC, (k_calbec_df<<<dim3(tilesp, tilesb, nsplit), 256, 0, c.stream>>>(
                                    nr, p.nproj, nb, kchunk, p.d_betar_df, xdf, part)));
  const int n = p.nproj * nb;
  HPSI_LAUNCH(c, HPSI_K_DSCALE,
              (k_dscale64r<<<(n + 255) / 256, 256, 0, c.stream>>>(p.nproj, nb, nsplit, part, p.d_rowptr, p.d_col,
                                                                  p.d_dvalr, w)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "Gamma-form double-float projection kernels launch");
  *wout = w;
  return HPSI_OK;
}

// w = D' <betar|x> of the real form in float64 (calbec and D-scale); *w points into the workspace.
int gamma_w_fp64(Context& c, const Problem& p, const void* x, bool x32, int nb, bool scaled, double** wout) {
  if (!p.d_betar) return fail(c, HPSI_EINVAL, "Gamma-form projectors are not prepared");
  const int nr = 2 * ((p.npw + 1) / 2);
  const int tilesp = (p.nproj + RB_TP - 1) / RB_TP, tilesb = (nb + RB_TB - 1) / RB_TB;
  int nsplit = std::max(1, (3 * c.sm_count) / std::max(1, tilesp * tilesb));
  int kchunk = (nr + nsplit - 1) / nsplit;
  kchunk = std::max(RB_TK * 2, ((kchunk + RB_TK - 1) / RB_TK) * RB_TK);
  nsplit = (nr + kchunk - 1) / kchunk;
  int rc = ensure_buffer(c, &c.ws.part, &c.ws.partbytes, sizeof(double) * (size_t)nsplit * nb * p.nproj);
  if (rc) return rc;
  rc = ensure_buffer(c, &c.ws.w, &c.ws.wbytes, sizeof(double) * (size_t)nb * p.nproj);
  if (rc) return rc;
  double* part = static_cast<double*>(c.ws.part);
  double* w = static_cast<double*>(c.ws.w);
  const dim3 gc(tilesp, tilesb, nsplit);
  if (x32)
    HPSI_LAUNCH(c, HPSI_K_CALBEC, (k_calbec64r<float><<<gc, 256, 0, c.stream>>>(
                                      nr, p.nproj, nb, kchunk, scaled ? 1 : 0, p.d_betar,
                                      static_cast<const float*>(x), part)));
  else
    HPSI_LAUNCH(c, HPSI_K_CALBEC, (k_calbec64r<double><<<gc, 256, 0, c.stream>>>(
                                      nr, p.nproj, nb, kchunk, scaled ? 1 : 0, p.d_betar,
                                      static_cast<const double*>(x), part)));
  const int n = p.nproj * nb;
  HPSI_LAUNCH(c, HPSI_K_DSCALE,
              (k_dscale64r<<<(n + 255) / 256, 256, 0, c.stream>>>(p.nproj, nb, nsplit, part, p.d_rowptr, p.d_col,
                                                                  p.d_dvalr, w)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "Gamma-form float64 projection kernels launch");
  *wout = w;
  return HPSI_OK;
}

int gamma_nonlocal_fp64(Context& c, const Problem& p, const void* x, bool x32, int nb, bool scaled, double* out) {
  if (p.nproj == 0 || nb == 0) return HPSI_OK;
  const int nr = 2 * ((p.npw + 1) / 2);
  double* w = nullptr;
  int rc = gamma_w_fp64(c, p, x, x32, nb, scaled, &w);
  if (rc) return rc;
  HPSI_LAUNCH(c, HPSI_K_ADDVUS,
              (k_addvus64r<<<dim3((nr + RA_TR - 1) / RA_TR, (nb + RA_TB - 1) / RA_TB), 256, 0, c.stream>>>(
                  nr, p.nproj, nb, w, p.d_betar, out)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "Gamma-form float64 nonlocal kernels launch");
  return HPSI_OK;
}

// w = D <beta|psi> of the complex form in float64 (calbec and D-scale); *w points into the workspace.
int nonlocal_w_fp64(Context& c, const Problem& p, const double2* psi, int nbnd, double2** wout) {
  const int tilesp = (p.nproj + CB_TP - 1) / CB_TP, tilesb = (nbnd + CB_TB - 1) / CB_TB;
  int nsplit = 0, kchunk = 0;
  size_t bytes = 0;
  nonlocal_fp64_plan(c, p, nbnd, &nsplit, &kchunk, &bytes);
  int rc = ensure_buffer(c, &c.ws.part, &c.ws.partbytes, sizeof(double2) * (size_t)nsplit * nbnd * p.nproj);
  if (rc) return rc;
  rc = ensure_buffer(c, &c.ws.w, &c.ws.wbytes, sizeof(double2) * (size_t)nbnd * p.nproj);
  if (rc) return rc;
  double2* part = reinterpret_cast<double2*>(c.ws.part);
  double2* w = reinterpret_cast<double2*>(c.ws.w);
  HPSI_LAUNCH(c, HPSI_K_CALBEC,
              (k_calbec64<<<dim3(tilesp, tilesb, nsplit), 256, 0, c.stream>>>(p.npw, p.nproj, nbnd, kchunk,
                                                                              p.d_beta, psi, part)));
  const int n = p.nproj * nbnd;
  HPSI_LAUNCH(c, HPSI_K_DSCALE,
              (k_dscale64<<<(n + 255) / 256, 256, 0, c.stream>>>(p.nproj, nbnd, nsplit, part, p.d_rowptr, p.d_col,
                                                                 p.d_dval, w)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "float64 projection kernels launch");
  *wout = w;
  return HPSI_OK;
}

int nonlocal_apply_fp64(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd) {
  if (p.nproj == 0 || nbnd == 0) return HPSI_OK;
  double2* w = nullptr;
  int rc = nonlocal_w_fp64(c, p, psi, nbnd, &w);
  if (rc) return rc;
  HPSI_LAUNCH(c, HPSI_K_ADDVUS,
              (k_addvus64<<<dim3((p.npw + AV_TG - 1) / AV_TG, (nbnd + AV_TB - 1) / AV_TB), 256, 0, c.stream>>>(
                  p.npw, p.nproj, nbnd, w, p.d_beta, hpsi)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "nonlocal float64 kernels launch");
  return HPSI_OK;
}

// Split of calbec's K = npw range for nbnd bands, and the partial / w bytes it needs.  With
// max_bytes > 0 the split count is lowered until the partials and w fit in max_bytes; *bytes is
// then still larger than max_bytes only if one split does not fit either (nsplit = 1).
void nonlocal_fp64_plan(const Context& c, const Problem& p, int nbnd, int* nsplit, int* kchunk, size_t* bytes,
                        size_t max_bytes) {
  const int tilesp = (p.nproj + CB_TP - 1) / CB_TP, tilesb = (nbnd + CB_TB - 1) / CB_TB;
  int ns = std::max(1, (3 * c.sm_count) / std::max(1, tilesp * tilesb));
  const size_t unit = sizeof(double2) * (size_t)nbnd * p.nproj;   // one split's partials, or w
  if (max_bytes > 0 && unit > 0) {
    const size_t cap = max_bytes / unit;                           // splits + 1 that fit
    ns = std::min<size_t>(ns, cap > 1 ? cap - 1 : 1);
  }
  int kc = (p.npw + ns - 1) / ns;
  kc = std::max(CB_TK * 4, ((kc + CB_TK - 1) / CB_TK) * CB_TK);
  ns = (p.npw + kc - 1) / kc;   // never above the ns that kc was derived from
  *nsplit = ns;
  *kchunk = kc;
  *bytes = unit * ((size_t)ns + 1);
}

// The same three launches with caller-provided partial and w buffers of `capacity` bytes; the
// K-split is planned to fit them (HPSI_EINVAL, before any launch, if even one split does not).
int nonlocal_fp64_into(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, void* scratch,
                       size_t capacity) {
  if (p.nproj == 0 || nbnd == 0) return HPSI_OK;
  int nsplit = 0, kchunk = 0;
  size_t bytes = 0;
  nonlocal_fp64_plan(c, p, nbnd, &nsplit, &kchunk, &bytes, capacity);
  if (bytes > capacity) return fail(c, HPSI_EINVAL, "nonlocal float64 kernels: partial sums do not fit the scratch");
  const int tilesp = (p.nproj + CB_TP - 1) / CB_TP, tilesb = (nbnd + CB_TB - 1) / CB_TB;
  double2* part = reinterpret_cast<double2*>(scratch);
  double2* w = part + (size_t)nsplit * nbnd * p.nproj;
  HPSI_LAUNCH(c, HPSI_K_CALBEC,
              (k_calbec64<<<dim3(tilesp, tilesb, nsplit), 256, 0, c.stream>>>(p.npw, p.nproj, nbnd, kchunk,
                                                                              p.d_beta, psi, part)));
  const int n = p.nproj * nbnd;
  HPSI_LAUNCH(c, HPSI_K_DSCALE,
              (k_dscale64<<<(n + 255) / 256, 256, 0, c.stream>>>(p.nproj, nbnd, nsplit, part, p.d_rowptr, p.d_col,
                                                                 p.d_dval, w)));
  HPSI_LAUNCH(c, HPSI_K_ADDVUS,
              (k_addvus64<<<dim3((p.npw + AV_TG - 1) / AV_TG, (nbnd + AV_TB - 1) / AV_TB), 256, 0, c.stream>>>(
                  p.npw, p.nproj, nbnd, w, p.d_beta, hpsi)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "nonlocal float64 kernels launch");
  return HPSI_OK;
}

// The float64 nonlocal term of several items in one launch per kernel class (groups of kNlBatch).
int nonlocal_batch_fp64(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                        double2* const* hpsi) {
  std::vector<int> items;
  for (int i = 0; i < nitem; ++i)
    if (nbnd[i] > 0 && c.probs[prob[i]].nproj > 0) items.push_back(i);
  // partial sums and w of every item side by side in one workspace
  std::vector<size_t> off(items.size());
  std::vector<int> ns(items.size()), kc(items.size());
  size_t total = 0;
  for (size_t j = 0; j < items.size(); ++j) {
    const Problem& p = c.probs[prob[items[j]]];
    size_t bytes = 0;
    nonlocal_fp64_plan(c, p, nbnd[items[j]], &ns[j], &kc[j], &bytes);
    off[j] = total;
    total += (bytes + 255) & ~size_t(255);
  }
  if (items.empty()) return HPSI_OK;
  int rc = ensure_buffer(c, &c.ws.part, &c.ws.partbytes, total);
  if (rc) return rc;
  unsigned char* base = static_cast<unsigned char*>(c.ws.part);
  static NlBatch bt;   // host staging of the parameter block (calls are not thread-safe by contract)
  for (size_t g0 = 0; g0 < items.size(); g0 += kNlBatch) {
    const int n = (int)std::min<size_t>(kNlBatch, items.size() - g0);
    bt.nitems = n;
    bt.off_cal[0] = bt.off_ds[0] = bt.off_add[0] = 0;
    for (int t = 0; t < n; ++t) {
      const size_t j = g0 + t;
      const int i = items[j];
      const Problem& p = c.probs[prob[i]];
      NlItem& a = bt.item[t];
      a.npw = p.npw;
      a.nproj = p.nproj;
      a.nb = nbnd[i];
      a.kchunk = kc[j];
      a.nsplit = ns[j];
      a.tp = calbec_tp(p.nproj);
      a.tilesp = (p.nproj + a.tp - 1) / a.tp;
      a.tilesb = (a.nb + CB_TB - 1) / CB_TB;
      a.gtiles = (p.npw + AV_TG - 1) / AV_TG;
      a.beta = p.d_beta;
      a.psi = psi[i];
      a.hpsi = hpsi[i];
      a.part = reinterpret_cast<double2*>(base + off[j]);
      a.w = a.part + (size_t)a.nsplit * a.nb * a.nproj;
      a.rowptr = p.d_rowptr;
      a.col = p.d_col;
      a.dval = p.d_dval;
      bt.off_cal[t + 1] = bt.off_cal[t] + a.tilesp * a.tilesb * a.nsplit;
      bt.off_ds[t + 1] = bt.off_ds[t] + (a.nproj * a.nb + 255) / 256;
      bt.off_add[t + 1] = bt.off_add[t] + a.gtiles * ((a.nb + AV_TB - 1) / AV_TB);
    }
    HPSI_LAUNCH(c, HPSI_K_CALBEC, (k_calbec64_batch<<<bt.off_cal[n], 256, 0, c.stream>>>(bt)));
    HPSI_LAUNCH(c, HPSI_K_DSCALE, (k_dscale64_batch<<<bt.off_ds[n], 256, 0, c.stream>>>(bt)));
    HPSI_LAUNCH(c, HPSI_K_ADDVUS, (k_addvus64_batch<<<bt.off_add[n], 256, 0, c.stream>>>(bt)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "batched float64 nonlocal kernels launch");
  }
  return HPSI_OK;
}

}  // namespace hpsi
