// Fast local part of H|psi> for cubic boxes whose edge N = R1 * R2 has register codelets.
//
// Three kernels per band block (App. A.1: V applied in real space between the two transforms):
//   k_zinv   per (band, chunk of sticks): scatter psi(G) into each z-stick (zero elsewhere), inverse
//            z-transform, stage the chunk in shared memory and write Zt[b][j3][stick] coalesced.
//   k_plane  per (z-plane j3, group of bands): per m1-plane an inverse y-transform of its sticks,
//            per j2 an inverse x-transform over the m1-planes, x V(r), forward x-transform keeping
//            the m1-planes, per m1-plane a forward y-transform keeping the sticks -> Y[b][j3][stick].
//            The plane [m1-plane][j2] lives in shared memory; nothing but the stick rows touches HBM.
//   k_zfwd   per (band, chunk of sticks): forward z-transform, keep the sphere, 1/N_r, add the
//            kinetic term |k+G|^2/2 psi(G) in float64.
// Each line transform is fft2_nat / fft2_rev (fft_codelets.cuh) on a group of max(R1, R2) threads.
#include <cuda_runtime.h>

#include <algorithm>

#include "fft_codelets.cuh"
#include "hpsi_internal.h"

namespace hpsi {

namespace {

struct FastArgs {
  int N, npw, npl, nst, nb, bpc;   // bpc: bands per k_plane CTA
  int stage_v, stage_row;
  const StickDev* sticks;
  const int* ymap;     // [npl][N]: stick of (plane, j2) or -1
  const int* xmap;     // [N]: plane of ix or -1
  const double2* psi;  // [nb][npw]
  double2* hpsi;
  const double* kin;
  void* Zt;            // [nb][N][nst]
  void* Yb;            // [nb][N][nst]
  const void* V;       // [N][N][N] as [j3][j2][j1]
  const double2* tw64; // e^{-2 pi i j / N}, j < N
  const float2* tw32;
  double inv_nr;
};

template <typename V> __device__ __forceinline__ const V* twt(const FastArgs& a);
template <> __device__ __forceinline__ const double2* twt<double2>(const FastArgs& a) { return a.tw64; }
template <> __device__ __forceinline__ const float2* twt<float2>(const FastArgs& a) { return a.tw32; }

template <typename V> __device__ __forceinline__ V d2v(double2 x);
template <> __device__ __forceinline__ double2 d2v<double2>(double2 x) { return x; }
template <> __device__ __forceinline__ float2 d2v<float2>(double2 x) { return make_float2((float)x.x, (float)x.y); }

template <int R1, int R2> struct Geo {
  static constexpr int N = R1 * R2;
  static constexpr int G = R1 > R2 ? R1 : R2;
  static constexpr int LPW = 32 / G;          // line groups per warp
  static constexpr int GROUPS = 8 * LPW;      // per 256-thread CTA
};

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256) k_zinv(FastArgs a) {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N, G = Gm::G, SC = Gm::GROUPS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* xbuf = tw + N;                       // [SC][N]
  V* obuf = xbuf + SC * N;                // [N][SC]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * Gm::LPW + lane / G, t = lane % G;
  const bool in_grp = lane < Gm::LPW * G;
  const int s0 = blockIdx.x * SC, b = blockIdx.y;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twt<V>(a)[i];
  __syncthreads();
  const int s = s0 + grp;
  const bool active = in_grp && s < a.nst;
  V reg[G];
  if (active && t < R2) {
    const StickDev st = a.sticks[s];
    const double2* ps = a.psi + (size_t)b * a.npw + st.g0;
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      int tt = R2 * n1 + t - st.z0;
      if (tt < 0) tt += N;
      reg[n1] = tt < st.len ? d2v<V>(ps[tt]) : czero<V>();
    }
  }
  fft2_nat<R1, R2, +1>(reg, xbuf + (in_grp ? grp : 0) * N, tw, t, active);
  if (active && t < R1) {
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) obuf[(t + R1 * k2) * SC + grp] = reg[k2];
  }
  __syncthreads();
  V* Z = reinterpret_cast<V*>(a.Zt) + (size_t)b * N * a.nst;
  const int ns = min(SC, a.nst - s0);
  for (int i = threadIdx.x; i < N * SC; i += blockDim.x) {
    const int j3 = i / SC, sl = i - j3 * SC;
    if (sl < ns) Z[(size_t)j3 * a.nst + s0 + sl] = obuf[i];
  }
}

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256) k_plane(FastArgs a) {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N, G = Gm::G, NG = Gm::GROUPS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* xbuf = tw + N;                              // [NG][N]
  V* P = xbuf + NG * N;                          // [npl][N]
  V* row = P + (size_t)a.npl * N;                // [nst] if stage_row
  T* vpl = reinterpret_cast<T*>(row + (a.stage_row ? a.nst : 0));   // [N][N] if stage_v
  int* xm = reinterpret_cast<int*>(vpl + (a.stage_v ? N * N : 0));  // [N]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * Gm::LPW + lane / G, t = lane % G;
  const bool in_grp = lane < Gm::LPW * G;
  V* xb = xbuf + (in_grp ? grp : 0) * N;
  const int j3 = blockIdx.x;
  const T* Vg = reinterpret_cast<const T*>(a.V) + (size_t)j3 * N * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tw[i] = twt<V>(a)[i];
    xm[i] = a.xmap[i];
  }
  if (a.stage_v)
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) vpl[i] = Vg[i];
  const T* Vp = a.stage_v ? vpl : Vg;
  for (int bi = 0; bi < a.bpc; ++bi) {
    const int b = blockIdx.y * a.bpc + bi;
    if (b >= a.nb) break;
    const V* zin = reinterpret_cast<const V*>(a.Zt) + ((size_t)b * N + j3) * a.nst;
    V* yout = reinterpret_cast<V*>(a.Yb) + ((size_t)b * N + j3) * a.nst;
    __syncthreads();
    if (a.stage_row)
      for (int i = threadIdx.x; i < a.nst; i += blockDim.x) row[i] = zin[i];
    __syncthreads();
    const V* src = a.stage_row ? row : zin;
    V reg[G];
    // inverse y per m1-plane: inputs at the plane's sticks
    for (int p0 = 0; p0 < a.npl; p0 += NG) {
      const int p = p0 + grp;
      const bool act = in_grp && p < a.npl;
      if (act && t < R2) {
        const int* ym = a.ymap + (size_t)p * N;
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
          const int s = __ldg(ym + R2 * n1 + t);
          reg[n1] = s >= 0 ? src[s] : czero<V>();
        }
      }
      fft2_nat<R1, R2, +1>(reg, xb, tw, t, act);
      if (act && t < R1) {
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) P[(size_t)p * N + t + R1 * k2] = reg[k2];
      }
    }
    __syncthreads();
    // x lines: inverse over the m1-planes, x V, forward keeping the m1-planes
    for (int q0 = 0; q0 < N; q0 += NG) {
      const int j2 = q0 + grp;
      const bool act = in_grp && j2 < N;
      if (act && t < R2) {
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
          const int pp = xm[R2 * n1 + t];
          reg[n1] = pp >= 0 ? P[(size_t)pp * N + j2] : czero<V>();
        }
      }
      fft2_nat<R1, R2, +1>(reg, xb, tw, t, act);
      if (act && t < R1) {
        const T* vr = Vp + (size_t)j2 * N;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) reg[k2] = cscale(reg[k2], vr[t + R1 * k2]);
      }
      fft2_rev<R1, R2, -1>(reg, xb, tw, t, act);
      if (act && t < R2) {
#pragma unroll
        for (int m1 = 0; m1 < R1; ++m1) {
          const int pp = xm[t + R2 * m1];
          if (pp >= 0) P[(size_t)pp * N + j2] = reg[m1];
        }
      }
    }
    __syncthreads();
    // forward y per m1-plane, keep the sticks
    V* dst = a.stage_row ? row : yout;
    for (int p0 = 0; p0 < a.npl; p0 += NG) {
      const int p = p0 + grp;
      const bool act = in_grp && p < a.npl;
      if (act && t < R2) {
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) reg[n1] = P[(size_t)p * N + R2 * n1 + t];
      }
      fft2_nat<R1, R2, -1>(reg, xb, tw, t, act);
      if (act && t < R1) {
        const int* ym = a.ymap + (size_t)p * N;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const int s = __ldg(ym + t + R1 * k2);
          if (s >= 0) dst[s] = reg[k2];
        }
      }
    }
    if (a.stage_row) {
      __syncthreads();
      for (int i = threadIdx.x; i < a.nst; i += blockDim.x) yout[i] = row[i];
    }
  }
}

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256) k_zfwd(FastArgs a) {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N, G = Gm::G, SC = Gm::GROUPS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* xbuf = tw + N;                       // [SC][N]
  V* ibuf = xbuf + SC * N;                // [N][SC]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * Gm::LPW + lane / G, t = lane % G;
  const bool in_grp = lane < Gm::LPW * G;
  const int s0 = blockIdx.x * SC, b = blockIdx.y;
  const int ns = min(SC, a.nst - s0);
  const V* Y = reinterpret_cast<const V*>(a.Yb) + (size_t)b * N * a.nst;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twt<V>(a)[i];
  for (int i = threadIdx.x; i < N * SC; i += blockDim.x) {
    const int j3 = i / SC, sl = i - j3 * SC;
    ibuf[i] = sl < ns ? Y[(size_t)j3 * a.nst + s0 + sl] : czero<V>();
  }
  __syncthreads();
  const int s = s0 + grp;
  const bool active = in_grp && s < a.nst;
  V reg[G];
  if (active && t < R2) {
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) reg[n1] = ibuf[(R2 * n1 + t) * SC + grp];
  }
  fft2_nat<R1, R2, -1>(reg, xbuf + (in_grp ? grp : 0) * N, tw, t, active);
  if (active && t < R1) {
    const StickDev st = a.sticks[s];
    const double2* ps = a.psi + (size_t)b * a.npw + st.g0;
    double2* out = a.hpsi + (size_t)b * a.npw + st.g0;
    const double* kin = a.kin + st.g0;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) {
      int tt = t + R1 * k2 - st.z0;
      if (tt < 0) tt += N;
      if (tt < st.len) {
        const double2 x = ps[tt];
        const double kg = kin[tt];
        const V v = reg[k2];
        out[tt] = make_double2(kg * x.x + (double)v.x * a.inv_nr, kg * x.y + (double)v.y * a.inv_nr);
      }
    }
  }
}

template <typename T, int R1, int R2>
struct FastKernels {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  static size_t smem_z() { return sizeof(V) * (size_t)(Gm::N + 2 * Gm::GROUPS * Gm::N); }
  static size_t smem_plane(const Problem& p, int sv, int sr) {
    return sizeof(V) * (size_t)(Gm::N + Gm::GROUPS * Gm::N + (size_t)p.npl * Gm::N + (sr ? p.nst : 0)) +
           (sv ? sizeof(T) * (size_t)Gm::N * Gm::N : 0) + sizeof(int) * Gm::N;
  }
  static int run(Context& c, const Problem& p, const FastArgs& a0, int nbnd, int nbb, int sv, int sr) {
    static bool attr = false;
    if (!attr) {
      const int mx = (int)c.smem_optin;
      cudaFuncSetAttribute(k_zinv<T, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      cudaFuncSetAttribute(k_plane<T, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      cudaFuncSetAttribute(k_zfwd<T, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      attr = true;
    }
    FastArgs a = a0;
    a.stage_v = sv;
    a.stage_row = sr;
    const size_t sz = smem_z(), sp = smem_plane(p, sv, sr);
    const int zch = (p.nst + Gm::GROUPS - 1) / Gm::GROUPS;
    for (int b0 = 0; b0 < nbnd; b0 += nbb) {
      const int nb = std::min(nbb, nbnd - b0);
      a.nb = nb;
      a.psi = a0.psi + (size_t)b0 * p.npw;
      a.hpsi = a0.hpsi + (size_t)b0 * p.npw;
      // bands per k_plane CTA: amortise the staged V plane while keeping >= 2 waves
      const int occ = sp <= c.smem_optin / 2 ? 2 : 1;
      int bpc = std::max(1, (Gm::N * nb) / (2 * c.sm_count * occ));
      bpc = std::min(bpc, 8);
      a.bpc = bpc;
      HPSI_LAUNCH(c, HPSI_K_INV_ZY, (k_zinv<T, R1, R2><<<dim3(zch, nb), 256, sz, c.stream>>>(a)));
      HPSI_LAUNCH(c, HPSI_K_XVX_Y,
                  (k_plane<T, R1, R2><<<dim3(Gm::N, (nb + bpc - 1) / bpc), 256, sp, c.stream>>>(a)));
      HPSI_LAUNCH(c, HPSI_K_FWD_Z, (k_zfwd<T, R1, R2><<<dim3(zch, nb), 256, sz, c.stream>>>(a)));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "fast local kernels launch");
    return HPSI_OK;
  }
};

// Factorisations N = R1 * R2 of the supported cubic edges.
template <typename T, typename F>
bool dispatch_size(int n, F&& f) {
  switch (n) {
    case 24: f(FastKernels<T, 4, 6>()); return true;
    case 25: f(FastKernels<T, 5, 5>()); return true;
    case 27: f(FastKernels<T, 3, 9>()); return true;
    case 30: f(FastKernels<T, 5, 6>()); return true;
    case 32: f(FastKernels<T, 4, 8>()); return true;
    case 36: f(FastKernels<T, 6, 6>()); return true;
    case 40: f(FastKernels<T, 5, 8>()); return true;
    case 45: f(FastKernels<T, 5, 9>()); return true;
    case 48: f(FastKernels<T, 6, 8>()); return true;
    case 50: f(FastKernels<T, 5, 10>()); return true;
    case 60: f(FastKernels<T, 6, 10>()); return true;
    case 64: f(FastKernels<T, 8, 8>()); return true;
    case 72: f(FastKernels<T, 8, 9>()); return true;
    case 80: f(FastKernels<T, 8, 10>()); return true;
    case 90: f(FastKernels<T, 9, 10>()); return true;
    case 96: f(FastKernels<T, 8, 12>()); return true;
    case 100: f(FastKernels<T, 10, 10>()); return true;
    case 120: f(FastKernels<T, 10, 12>()); return true;
    case 128: f(FastKernels<T, 8, 16>()); return true;
    case 144: f(FastKernels<T, 12, 12>()); return true;
    default: return false;
  }
}

}  // namespace

// Shared-memory plan of the fast path for a problem (0 if the box has no fast kernels or the
// plane does not fit): bit 0 stage V, bit 1 stage the stick row, bit 2 supported.
int local_fast_plan(const Problem& p, int precision, size_t smem_optin) {
  if (p.n[0] != p.n[1] || p.n[1] != p.n[2]) return 0;
  int flags = 0;
  auto pick = [&](auto k) {
    using K = decltype(k);
    for (int cand : {3, 2, 0}) {
      const int sv = cand & 1, sr = (cand >> 1) & 1;
      if (K::smem_z() <= smem_optin && K::smem_plane(p, sv, sr) <= smem_optin) {
        flags = 4 | sv | (sr << 1);
        return;
      }
    }
  };
  if (precision == HPSI_FP64) dispatch_size<double>(p.n[0], pick);
  else dispatch_size<float>(p.n[0], pick);
  return flags;
}

int local_fast_apply(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, void* Zt, void* Yb,
                     int nbb) {
  const int flags = p.fast_flags;
  FastArgs a;
  a.N = p.n[0];
  a.npw = p.npw;
  a.npl = p.npl;
  a.nst = p.nst;
  a.sticks = p.d_sticks;
  a.ymap = p.d_ymap;
  a.xmap = p.d_xmap;
  a.psi = psi;
  a.hpsi = hpsi;
  a.kin = p.d_kin;
  a.Zt = Zt;
  a.Yb = Yb;
  a.V = c.precision == HPSI_FP64 ? (const void*)p.d_v64 : (const void*)p.d_v32;
  a.tw64 = p.d_ftw64;
  a.tw32 = p.d_ftw32;
  a.inv_nr = 1.0 / ((double)p.n[0] * p.n[1] * p.n[2]);
  int rc = HPSI_EINVAL;
  auto go = [&](auto k) { rc = decltype(k)::run(c, p, a, nbnd, nbb, flags & 1, (flags >> 1) & 1); };
  if (c.precision == HPSI_FP64) dispatch_size<double>(p.n[0], go);
  else dispatch_size<float>(p.n[0], go);
  return rc;
}

}  // namespace hpsi
