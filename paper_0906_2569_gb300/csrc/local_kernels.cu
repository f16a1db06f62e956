// Local part of H|psi>: kinetic diagonal + [V psi](G) through sphere-pruned 3-D FFTs.
//
// The paper applies V(r) in real space with FFTs between the PW and grid representations
// (App. A.1; FFT layer of Sec. 2).  Here the 3-D transform is split by what each stage needs:
//
//   k_inv_zy   one CTA per (band, m1-plane): scatter psi(G) of the plane's sticks into
//              shared memory (zero elsewhere), inverse z-FFT of every stick, then for every
//              z-row an inverse y-FFT over the plane (only the plane's m2 entries are non-zero);
//              writes X[b][j3][plane][j2].
//   k_xvx_y    one CTA per (band, j3): for each j2 an inverse x-FFT over the m1-planes (only
//              those entries non-zero), x V(r), forward x-FFT keeping the plane entries; then a
//              forward y-FFT per plane keeping the sticks; writes Y[b][j3][stick].
//   k_fwd_z    one CTA per (band, m1-plane): forward z-FFT of the plane's sticks, keep the
//              sphere entries, scale by 1/N_r and add |k+G|^2/2 psi(G) (float64); writes hpsi.
//
// T = double is the float64 path; T = float keeps X, Y, V and the transforms in float32 while
// psi, the kinetic term and hpsi stay float64.  The full box never exists in memory: X holds
// only the m1-planes that carry sticks, Y only the sticks.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "hpsi_internal.h"
#include "warp_fft.cuh"

namespace hpsi {

struct LocalArgs {
  int n1, n2, n3, npw, npl, nst, ns_max, nb;
  const StickDev* sticks;
  const PlaneDev* planes;
  const double2* psi;   // [nb][npw]
  double2* hpsi;        // [nb][npw]
  const double* kin;    // [npw]
  void* X;              // [nb][n3][npl][n2]
  void* Y;              // [nb][n3][nst]
  const void* V;        // [n3][n2][n1]
  FftPlan p1, p2, p3;
  double inv_nr;
};

template <typename V> __device__ __forceinline__ V from_d2(double2 a);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}

template <typename T>
__global__ void __launch_bounds__(256) k_inv_zy(LocalArgs a) {
  using V = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* S = reinterpret_cast<V*>(smem_raw);             // [ns][n3]
  V* L = S + (size_t)a.ns_max * a.n3;                // [8][n2]
  int* iy = reinterpret_cast<int*>(L + kWarpsPerCta * a.n2);   // [ns]
  const int p = blockIdx.x, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const PlaneDev pl = a.planes[p];
  const int n3 = a.n3, n2 = a.n2;
  for (int i = threadIdx.x; i < pl.ns * n3; i += blockDim.x) S[i] = czero<V>();
  for (int s = threadIdx.x; s < pl.ns; s += blockDim.x) iy[s] = a.sticks[pl.s0 + s].iy;
  __syncthreads();
  const double2* psi = a.psi + (size_t)b * a.npw;
  for (int s = warp; s < pl.ns; s += kWarpsPerCta) {
    const StickDev st = a.sticks[pl.s0 + s];
    for (int t = lane; t < st.len; t += 32) {
      int z = st.z0 + t;
      if (z >= n3) z -= n3;
      S[s * n3 + z] = from_d2<V>(psi[st.g0 + t]);
    }
  }
  __syncthreads();
  for (int s = warp; s < pl.ns; s += kWarpsPerCta) warp_fft<+1>(S + s * n3, a.p3, lane);
  __syncthreads();
  V* Lw = L + warp * n2;
  V* X = reinterpret_cast<V*>(a.X) + (size_t)b * n3 * a.npl * n2;
  for (int j3 = warp; j3 < n3; j3 += kWarpsPerCta) {
    for (int i = lane; i < n2; i += 32) Lw[i] = czero<V>();
    __syncwarp();
    for (int s = lane; s < pl.ns; s += 32) Lw[iy[s]] = S[s * n3 + j3];
    __syncwarp();
    warp_fft<+1>(Lw, a.p2, lane);
    V* dst = X + ((size_t)j3 * a.npl + p) * n2;
    for (int i = lane; i < n2; i += 32) dst[i] = Lw[i];
    __syncwarp();
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_xvx_y(LocalArgs a) {
  using V = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* P = reinterpret_cast<V*>(smem_raw);             // [npl][n2]
  V* L = P + (size_t)a.npl * a.n2;                   // [8][n1]
  int* ix = reinterpret_cast<int*>(L + kWarpsPerCta * a.n1);   // [npl]
  const int j3 = blockIdx.x, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n1 = a.n1, n2 = a.n2, npl = a.npl;
  const V* X = reinterpret_cast<const V*>(a.X) + ((size_t)b * a.n3 + j3) * npl * n2;
  for (int i = threadIdx.x; i < npl * n2; i += blockDim.x) P[i] = X[i];
  for (int q = threadIdx.x; q < npl; q += blockDim.x) ix[q] = a.planes[q].ix;
  __syncthreads();
  const T* Vrow0 = reinterpret_cast<const T*>(a.V) + (size_t)j3 * n2 * n1;
  V* Lw = L + warp * n1;
  for (int j2 = warp; j2 < n2; j2 += kWarpsPerCta) {
    for (int i = lane; i < n1; i += 32) Lw[i] = czero<V>();
    __syncwarp();
    for (int q = lane; q < npl; q += 32) Lw[ix[q]] = P[q * n2 + j2];
    __syncwarp();
    warp_fft<+1>(Lw, a.p1, lane);
    const T* vr = Vrow0 + (size_t)j2 * n1;
    for (int i = lane; i < n1; i += 32) Lw[i] = cscale(Lw[i], __ldg(vr + i));
    __syncwarp();
    warp_fft<-1>(Lw, a.p1, lane);
    for (int q = lane; q < npl; q += 32) P[q * n2 + j2] = Lw[ix[q]];
    __syncwarp();
  }
  __syncthreads();
  V* Y = reinterpret_cast<V*>(a.Y) + ((size_t)b * a.n3 + j3) * a.nst;
  for (int q = warp; q < npl; q += kWarpsPerCta) {
    V* line = P + q * n2;
    warp_fft<-1>(line, a.p2, lane);
    const PlaneDev pl = a.planes[q];
    for (int s = lane; s < pl.ns; s += 32) Y[pl.s0 + s] = line[a.sticks[pl.s0 + s].iy];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fwd_z(LocalArgs a) {
  using V = typename Cx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* S = reinterpret_cast<V*>(smem_raw);             // [ns][n3]
  const int p = blockIdx.x, b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const PlaneDev pl = a.planes[p];
  const int n3 = a.n3;
  const V* Y = reinterpret_cast<const V*>(a.Y) + (size_t)b * n3 * a.nst + pl.s0;
  for (int i = threadIdx.x; i < pl.ns * n3; i += blockDim.x) {
    const int j3 = i / pl.ns, s = i - j3 * pl.ns;
    S[s * n3 + j3] = Y[(size_t)j3 * a.nst + s];
  }
  __syncthreads();
  for (int s = warp; s < pl.ns; s += kWarpsPerCta) warp_fft<-1>(S + s * n3, a.p3, lane);
  __syncthreads();
  const double2* psi = a.psi + (size_t)b * a.npw;
  double2* out = a.hpsi + (size_t)b * a.npw;
  for (int s = warp; s < pl.ns; s += kWarpsPerCta) {
    const StickDev st = a.sticks[pl.s0 + s];
    for (int t = lane; t < st.len; t += 32) {
      int z = st.z0 + t;
      if (z >= n3) z -= n3;
      const V v = S[s * n3 + z];
      const int g = st.g0 + t;
      const double2 x = psi[g];
      const double kg = a.kin[g];
      out[g] = make_double2(kg * x.x + (double)v.x * a.inv_nr, kg * x.y + (double)v.y * a.inv_nr);
    }
  }
}

// Density of the orbitals on the grid (App. A.1, rho = sum_i f_i |psi_i(r)|^2): one CTA per j3 takes
// every band of the block in turn, inverse x-transforms its m1-plane entries (X, from k_inv_zy) and
// adds wb[b] |psi_b(r)|^2 into rho[j3][j2][j1].  Element (j3, j2, j1) is only ever touched by CTA
// j3, warp j2 mod 8, lane j1 mod 32, so the bands are summed in order without atomics.
__global__ void __launch_bounds__(256) k_x_density(LocalArgs a, const double* __restrict__ wb,
                                                   double* __restrict__ rho) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* P = reinterpret_cast<double2*>(smem_raw);       // [npl][n2]
  double2* L = P + (size_t)a.npl * a.n2;                   // [8][n1]
  int* ix = reinterpret_cast<int*>(L + kWarpsPerCta * a.n1);   // [npl]
  const int j3 = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n1 = a.n1, n2 = a.n2, npl = a.npl;
  for (int q = threadIdx.x; q < npl; q += blockDim.x) ix[q] = a.planes[q].ix;
  double2* Lw = L + warp * n1;
  for (int b = 0; b < a.nb; ++b) {
    __syncthreads();
    const double2* X = reinterpret_cast<const double2*>(a.X) + ((size_t)b * a.n3 + j3) * npl * n2;
    for (int i = threadIdx.x; i < npl * n2; i += blockDim.x) P[i] = X[i];
    __syncthreads();
    const double w = wb[b];
    for (int j2 = warp; j2 < n2; j2 += kWarpsPerCta) {
      for (int i = lane; i < n1; i += 32) Lw[i] = czero<double2>();
      __syncwarp();
      for (int q = lane; q < npl; q += 32) Lw[ix[q]] = P[q * n2 + j2];
      __syncwarp();
      warp_fft<+1>(Lw, a.p1, lane);
      double* row = rho + ((size_t)j3 * n2 + j2) * n1;
      for (int i = lane; i < n1; i += 32) row[i] += w * (Lw[i].x * Lw[i].x + Lw[i].y * Lw[i].y);
      __syncwarp();
    }
  }
}

// rho[j3][j2][j1] += sum_b wb[b] |psi_b(r_j)|^2 for nbnd float64 bands (wb on the device).
int local_density(Context& c, const Problem& p, const double2* psi, int nbnd, const double* wb, double* rho) {
  if (nbnd == 0) return HPSI_OK;
  const int nbb = std::max(1, std::min(p.nbb[HPSI_FP64], nbnd));
  const size_t xneed = sizeof(double2) * (size_t)nbb * p.n[2] * p.npl * p.n[1];
  int rc = ensure_buffer(c, &c.ws.X, &c.ws.xbytes, xneed);
  if (rc) return rc;
  const size_t s0 = local_smem_bytes(p, HPSI_FP64, 0), s1 = local_smem_bytes(p, HPSI_FP64, 1);
  const int mx = (int)c.smem_optin;
  cudaFuncSetAttribute(k_inv_zy<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_x_density, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  LocalArgs a;
  a.n1 = p.n[0]; a.n2 = p.n[1]; a.n3 = p.n[2];
  a.npw = p.npw; a.npl = p.npl; a.nst = p.nst; a.ns_max = p.ns_max;
  a.sticks = p.d_sticks; a.planes = p.d_planes; a.kin = p.d_kin;
  a.X = c.ws.X; a.Y = nullptr; a.V = nullptr; a.hpsi = nullptr;
  a.p1 = p.plan[0]; a.p2 = p.plan[1]; a.p3 = p.plan[2];
  a.inv_nr = 1.0 / ((double)p.n[0] * p.n[1] * p.n[2]);
  for (int b0 = 0; b0 < nbnd; b0 += nbb) {
    const int nb = std::min(nbb, nbnd - b0);
    a.nb = nb;
    a.psi = psi + (size_t)b0 * p.npw;
    HPSI_LAUNCH(c, HPSI_K_SCF, (k_inv_zy<double><<<dim3(p.npl, nb), 256, s0, c.stream>>>(a)));
    HPSI_LAUNCH(c, HPSI_K_SCF, (k_x_density<<<p.n[2], 256, s1, c.stream>>>(a, wb + b0, rho)));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "density kernels launch");
  return HPSI_OK;
}

// Shared memory of each kernel (bytes) for a problem at a precision; which = 0, 1, 2.
size_t local_smem_bytes(const Problem& p, int precision, int which) {
  const size_t cs = precision == HPSI_FP64 ? sizeof(double2) : sizeof(float2);
  if (which == 0)
    return cs * ((size_t)p.ns_max * p.n[2] + (size_t)kWarpsPerCta * p.n[1]) + sizeof(int) * p.ns_max;
  if (which == 1)
    return cs * ((size_t)p.npl * p.n[1] + (size_t)kWarpsPerCta * p.n[0]) + sizeof(int) * p.npl;
  return cs * (size_t)p.ns_max * p.n[2];
}

// Autotuner of the fast path: time every plan that fits the shared memory (which of the V plane
// and the stick row the plane kernel stages) against band blocks of half, one and two times the
// default, on this call's own bands, and keep the fastest.  Neither choice changes the arithmetic.
static int tune_fast(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, size_t cs) {
  const int pr = cur_prec(c);
  const std::vector<int> plans = local_fast_candidates(p, pr, c.smem_optin);
  const int nb0 = p.nbbf[pr];
  std::vector<int> blocks;
  for (int nb : {std::max(1, nb0 / 2), nb0, 2 * nb0}) {
    const int v = std::min(nb, nbnd);
    if (std::find(blocks.begin(), blocks.end(), v) == blocks.end()) blocks.push_back(v);
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return HPSI_OK;
  }
  float best = 1e30f;
  int best_plan = p.fflags[pr], best_nb = nb0;
  const bool timing = c.timing;
  c.timing = false;
  int rc = HPSI_OK;
  for (int plan : plans)
    for (int nb : blocks) {
      const size_t need = cs * (size_t)nb * p.n[2] * p.nst;
      rc = ensure_buffer(c, &c.ws.X, &c.ws.xbytes, need);
      if (!rc) rc = ensure_buffer(c, &c.ws.Y, &c.ws.ybytes, need);
      if (rc) break;
      p.fflags[pr] = plan;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && !rc; ++rep) {   // first run warms up, second is timed
        cudaEventRecord(e0, c.stream);
        rc = local_fast_apply(c, p, psi, hpsi, nbnd, c.ws.X, c.ws.Y, nb);
        cudaEventRecord(e1, c.stream);
      }
      if (rc) break;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) {
        best = ms;
        best_plan = plan;
        best_nb = nb;
      }
    }
  c.timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p.fflags[pr] = best_plan;
  p.nbbf[pr] = best_nb;
  p.tuned[pr] = true;
  return rc;
}

template <typename T>
static int local_apply_t(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd) {
  const size_t cs = sizeof(typename Cx<T>::type);
  if ((p.fflags[cur_prec(c)] & 4) && !c.force_generic) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c.stream, &cap);
    if (c.autotune && !p.tuned[cur_prec(c)] && nbnd >= 4 && cap == cudaStreamCaptureStatusNone) {
      int rc = tune_fast(c, p, psi, hpsi, nbnd, cs);
      if (rc) return rc;
    }
    const int nbf = std::max(1, std::min(p.nbbf[cur_prec(c)], nbnd));
    const size_t zneed = cs * (size_t)nbf * p.n[2] * p.nst;
    int rc = ensure_buffer(c, &c.ws.X, &c.ws.xbytes, zneed);
    if (rc) return rc;
    rc = ensure_buffer(c, &c.ws.Y, &c.ws.ybytes, zneed);
    if (rc) return rc;
    return local_fast_apply(c, p, psi, hpsi, nbnd, c.ws.X, c.ws.Y, nbf);
  }
  const int nbb = std::max(1, std::min(p.nbb[cur_prec(c)], nbnd));
  const size_t xneed = cs * (size_t)nbb * p.n[2] * p.npl * p.n[1];
  const size_t yneed = cs * (size_t)nbb * p.n[2] * p.nst;
  int rc = ensure_buffer(c, &c.ws.X, &c.ws.xbytes, xneed);
  if (rc) return rc;
  rc = ensure_buffer(c, &c.ws.Y, &c.ws.ybytes, yneed);
  if (rc) return rc;
  const size_t s0 = local_smem_bytes(p, cur_prec(c), 0), s1 = local_smem_bytes(p, cur_prec(c), 1),
               s2 = local_smem_bytes(p, cur_prec(c), 2);
  static bool attr_done[2] = {false, false};
  const int slot = sizeof(T) == 8 ? 0 : 1;
  if (!attr_done[slot]) {
    const int mx = (int)c.smem_optin;
    cudaFuncSetAttribute(k_inv_zy<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_xvx_y<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_fwd_z<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    attr_done[slot] = true;
  }
  LocalArgs a;
  a.n1 = p.n[0]; a.n2 = p.n[1]; a.n3 = p.n[2];
  a.npw = p.npw; a.npl = p.npl; a.nst = p.nst; a.ns_max = p.ns_max;
  a.sticks = p.d_sticks; a.planes = p.d_planes; a.kin = p.d_kin;
  a.X = c.ws.X; a.Y = c.ws.Y;
  a.V = sizeof(T) == 8 ? (const void*)p.d_v64 : (const void*)p.d_v32;
  a.p1 = p.plan[0]; a.p2 = p.plan[1]; a.p3 = p.plan[2];
  a.inv_nr = 1.0 / ((double)p.n[0] * p.n[1] * p.n[2]);
  for (int b0 = 0; b0 < nbnd; b0 += nbb) {
    const int nb = std::min(nbb, nbnd - b0);
    a.nb = nb;
    a.psi = psi + (size_t)b0 * p.npw;
    a.hpsi = hpsi + (size_t)b0 * p.npw;
    HPSI_LAUNCH(c, HPSI_K_INV_ZY, (k_inv_zy<T><<<dim3(p.npl, nb), 256, s0, c.stream>>>(a)));
    HPSI_LAUNCH(c, HPSI_K_XVX_Y, (k_xvx_y<T><<<dim3(p.n[2], nb), 256, s1, c.stream>>>(a)));
    HPSI_LAUNCH(c, HPSI_K_FWD_Z, (k_fwd_z<T><<<dim3(p.npl, nb), 256, s2, c.stream>>>(a)));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "local-potential kernels launch");
  return HPSI_OK;
}

int local_apply(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd) {
  if (cur_prec(c) == HPSI_FP64) return local_apply_t<double>(c, p, psi, hpsi, nbnd);
  return local_apply_t<float>(c, p, psi, hpsi, nbnd);
}

// Bytes of X and Y that one band needs at the context's precision.
size_t local_scratch_per_band(const Problem& p, int precision) {
  const size_t cs = precision == HPSI_FP64 ? sizeof(double2) : sizeof(float2);
  return cs * ((size_t)p.n[2] * p.npl * p.n[1] + (size_t)p.n[2] * p.nst);
}

// The same launch sequence with caller-provided X and Y (each sized for nbb bands).
template <typename T>
static int local_apply_into_t(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, void* X,
                              void* Y, int nbb) {
  const int mx = (int)c.smem_optin;
  cudaFuncSetAttribute(k_inv_zy<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_xvx_y<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  cudaFuncSetAttribute(k_fwd_z<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  const size_t s0 = local_smem_bytes(p, cur_prec(c), 0), s1 = local_smem_bytes(p, cur_prec(c), 1),
               s2 = local_smem_bytes(p, cur_prec(c), 2);
  LocalArgs a;
  a.n1 = p.n[0]; a.n2 = p.n[1]; a.n3 = p.n[2];
  a.npw = p.npw; a.npl = p.npl; a.nst = p.nst; a.ns_max = p.ns_max;
  a.sticks = p.d_sticks; a.planes = p.d_planes; a.kin = p.d_kin;
  a.X = X; a.Y = Y;
  a.V = sizeof(T) == 8 ? (const void*)p.d_v64 : (const void*)p.d_v32;
  a.p1 = p.plan[0]; a.p2 = p.plan[1]; a.p3 = p.plan[2];
  a.inv_nr = 1.0 / ((double)p.n[0] * p.n[1] * p.n[2]);
  for (int b0 = 0; b0 < nbnd; b0 += nbb) {
    const int nb = std::min(nbb, nbnd - b0);
    a.nb = nb;
    a.psi = psi + (size_t)b0 * p.npw;
    a.hpsi = hpsi + (size_t)b0 * p.npw;
    HPSI_LAUNCH(c, HPSI_K_INV_ZY, (k_inv_zy<T><<<dim3(p.npl, nb), 256, s0, c.stream>>>(a)));
    HPSI_LAUNCH(c, HPSI_K_XVX_Y, (k_xvx_y<T><<<dim3(p.n[2], nb), 256, s1, c.stream>>>(a)));
    HPSI_LAUNCH(c, HPSI_K_FWD_Z, (k_fwd_z<T><<<dim3(p.npl, nb), 256, s2, c.stream>>>(a)));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "local-potential kernels launch");
  return HPSI_OK;
}

int local_apply_into(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, void* X, void* Y,
                     int nbb) {
  if (cur_prec(c) == HPSI_FP64) return local_apply_into_t<double>(c, p, psi, hpsi, nbnd, X, Y, nbb);
  return local_apply_into_t<float>(c, p, psi, hpsi, nbnd, X, Y, nbb);
}

}  // namespace hpsi
