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

// One problem's share of a launch (a k-point or a cell with its band block).
struct FastItem {
  int nb, npw, npl, nst, bpc;  // bpc: bands per k_plane CTA
  const StickDev* sticks;
  const int* ymap;     // [npl][N]: stick of (plane, j2) or -1
  const int* xmap;     // [N]: plane of ix or -1
  const double2* psi;  // [nb][npw]
  double2* hpsi;
  const double* kin;
  void* Zt;            // [nb][N][nst]
  void* Yb;            // [nb][N][nst]
  const void* V;       // [N][N][N] as [j3][j2][j1]
};

constexpr int kMaxItems = 32;

// Every launch takes its items by value (the parameter block is 32 KB on sm_70 and later).
struct FastBatch {
  int nitems, N, stage_v, stage_row;
  const double2* tw64; // e^{-2 pi i j / N}, j < N
  const float2* tw32;
  double inv_nr;
  FastItem item[kMaxItems];
};

template <typename V> __device__ __forceinline__ const V* twt(const FastBatch& a);
template <> __device__ __forceinline__ const double2* twt<double2>(const FastBatch& a) { return a.tw64; }
template <> __device__ __forceinline__ const float2* twt<float2>(const FastBatch& a) { return a.tw32; }

template <typename V> __device__ __forceinline__ V d2v(double2 x);
template <> __device__ __forceinline__ double2 d2v<double2>(double2 x) { return x; }
template <> __device__ __forceinline__ float2 d2v<float2>(double2 x) { return make_float2((float)x.x, (float)x.y); }

template <int R1, int R2> struct Geo {
  static constexpr int N = R1 * R2;
  static constexpr int G = R1 > R2 ? R1 : R2;
  static constexpr int LPW = 32 / G;          // line groups per warp
  static constexpr int GROUPS = 8 * LPW;      // per 256-thread CTA
  static constexpr int XS = Xch<R1, R2>::size; // exchange-buffer entries per group
  static constexpr int PS = N + 1;            // row stride of the plane array (one pad entry)
};

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256) k_zinv(const __grid_constant__ FastBatch bt) {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N, G = Gm::G, SC = Gm::GROUPS;
  const FastItem& a = bt.item[blockIdx.z];
  if ((int)blockIdx.x * SC >= a.nst || (int)blockIdx.y >= a.nb) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* xbuf = tw + N;                       // [SC][XS]
  V* obuf = xbuf + SC * Gm::XS;           // [N][SC]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * Gm::LPW + lane / G, t = lane % G;
  const bool in_grp = lane < Gm::LPW * G;
  const int s0 = blockIdx.x * SC, b = blockIdx.y;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twt<V>(bt)[i];
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
  fft2_nat<R1, R2, +1>(reg, xbuf + (in_grp ? grp : 0) * Gm::XS, tw, t, active);
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
__global__ void __launch_bounds__(256) k_plane(const __grid_constant__ FastBatch bt) {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N, G = Gm::G, NG = Gm::GROUPS;
  const FastItem& a = bt.item[blockIdx.z];
  if ((int)blockIdx.y * a.bpc >= a.nb) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  constexpr int PS = Gm::PS;
  V* xbuf = tw + N;                              // [NG][XS]
  V* P = xbuf + NG * Gm::XS;                     // [npl][PS]
  V* row = P + (size_t)a.npl * PS;               // [nst] if stage_row
  T* vpl = reinterpret_cast<T*>(row + (bt.stage_row ? a.nst : 0));   // [N][N] if stage_v
  int* xm = reinterpret_cast<int*>(vpl + (bt.stage_v ? N * N : 0));  // [N]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * Gm::LPW + lane / G, t = lane % G;
  const bool in_grp = lane < Gm::LPW * G;
  V* xb = xbuf + (in_grp ? grp : 0) * Gm::XS;
  const int j3 = blockIdx.x;
  const T* Vg = reinterpret_cast<const T*>(a.V) + (size_t)j3 * N * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tw[i] = twt<V>(bt)[i];
    xm[i] = a.xmap[i];
  }
  if (bt.stage_v)
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) vpl[i] = Vg[i];
  const T* Vp = bt.stage_v ? vpl : Vg;
  for (int bi = 0; bi < a.bpc; ++bi) {
    const int b = blockIdx.y * a.bpc + bi;
    if (b >= a.nb) break;
    const V* zin = reinterpret_cast<const V*>(a.Zt) + ((size_t)b * N + j3) * a.nst;
    V* yout = reinterpret_cast<V*>(a.Yb) + ((size_t)b * N + j3) * a.nst;
    __syncthreads();
    if (bt.stage_row)
      for (int i = threadIdx.x; i < a.nst; i += blockDim.x) row[i] = zin[i];
    __syncthreads();
    const V* src = bt.stage_row ? row : zin;
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
        for (int k2 = 0; k2 < R2; ++k2) P[(size_t)p * PS + t + R1 * k2] = reg[k2];
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
          reg[n1] = pp >= 0 ? P[(size_t)pp * PS + j2] : czero<V>();
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
          if (pp >= 0) P[(size_t)pp * PS + j2] = reg[m1];
        }
      }
    }
    __syncthreads();
    // forward y per m1-plane, keep the sticks
    V* dst = bt.stage_row ? row : yout;
    for (int p0 = 0; p0 < a.npl; p0 += NG) {
      const int p = p0 + grp;
      const bool act = in_grp && p < a.npl;
      if (act && t < R2) {
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) reg[n1] = P[(size_t)p * PS + R2 * n1 + t];
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
    if (bt.stage_row) {
      __syncthreads();
      for (int i = threadIdx.x; i < a.nst; i += blockDim.x) yout[i] = row[i];
    }
  }
}

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256) k_zfwd(const __grid_constant__ FastBatch bt) {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N, G = Gm::G, SC = Gm::GROUPS;
  const FastItem& a = bt.item[blockIdx.z];
  if ((int)blockIdx.x * SC >= a.nst || (int)blockIdx.y >= a.nb) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* xbuf = tw + N;                       // [SC][XS]
  V* ibuf = xbuf + SC * Gm::XS;           // [N][SC]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * Gm::LPW + lane / G, t = lane % G;
  const bool in_grp = lane < Gm::LPW * G;
  const int s0 = blockIdx.x * SC, b = blockIdx.y;
  const int ns = min(SC, a.nst - s0);
  const V* Y = reinterpret_cast<const V*>(a.Yb) + (size_t)b * N * a.nst;
  for (int i = threadIdx.x; i < N; i += blockDim.x) tw[i] = twt<V>(bt)[i];
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
  fft2_nat<R1, R2, -1>(reg, xbuf + (in_grp ? grp : 0) * Gm::XS, tw, t, active);
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
        out[tt] = make_double2(kg * x.x + (double)v.x * bt.inv_nr, kg * x.y + (double)v.y * bt.inv_nr);
      }
    }
  }
}

template <typename T, int R1, int R2>
struct FastKernels {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  static size_t smem_z() { return sizeof(V) * (size_t)(Gm::N + Gm::GROUPS * Gm::XS + Gm::GROUPS * Gm::N); }
  static size_t smem_plane(const Problem& p, int sv, int sr) {
    return sizeof(V) * (size_t)(Gm::N + Gm::GROUPS * Gm::XS + (size_t)p.npl * Gm::PS + (sr ? p.nst : 0)) +
           (sv ? sizeof(T) * (size_t)Gm::N * Gm::N : 0) + sizeof(int) * Gm::N;
  }
  // One launch of each kernel over every item of the batch (all share the edge N and the flags).
  static int run(Context& c, FastBatch& bt, size_t max_plane_smem) {
    static bool attr = false;
    if (!attr) {
      const int mx = (int)c.smem_optin;
      cudaFuncSetAttribute(k_zinv<T, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      cudaFuncSetAttribute(k_plane<T, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      cudaFuncSetAttribute(k_zfwd<T, R1, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      attr = true;
    }
    const size_t sz = smem_z();
    int zch = 1, nbmax = 1, pyb = 1, total_rows = 0;
    for (int i = 0; i < bt.nitems; ++i) {
      FastItem& it = bt.item[i];
      zch = std::max(zch, (it.nst + Gm::GROUPS - 1) / Gm::GROUPS);
      nbmax = std::max(nbmax, it.nb);
      total_rows += it.nb;
    }
    // bands per k_plane CTA: amortise the staged V plane while keeping >= 2 waves over the batch
    const int occ = max_plane_smem <= c.smem_optin / 2 ? 2 : 1;
    int bpc = std::max(1, (Gm::N * total_rows) / (2 * c.sm_count * occ));
    bpc = std::min(bpc, 8);
    for (int i = 0; i < bt.nitems; ++i) {
      bt.item[i].bpc = bpc;
      pyb = std::max(pyb, (bt.item[i].nb + bpc - 1) / bpc);
    }
    HPSI_LAUNCH(c, HPSI_K_INV_ZY, (k_zinv<T, R1, R2><<<dim3(zch, nbmax, bt.nitems), 256, sz, c.stream>>>(bt)));
    HPSI_LAUNCH(c, HPSI_K_XVX_Y,
                (k_plane<T, R1, R2><<<dim3(Gm::N, pyb, bt.nitems), 256, max_plane_smem, c.stream>>>(bt)));
    HPSI_LAUNCH(c, HPSI_K_FWD_Z, (k_zfwd<T, R1, R2><<<dim3(zch, nbmax, bt.nitems), 256, sz, c.stream>>>(bt)));
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

static FastItem make_item(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nb, void* Zt, void* Yb) {
  FastItem it;
  it.nb = nb;
  it.npw = p.npw;
  it.npl = p.npl;
  it.nst = p.nst;
  it.bpc = 1;
  it.sticks = p.d_sticks;
  it.ymap = p.d_ymap;
  it.xmap = p.d_xmap;
  it.psi = psi;
  it.hpsi = hpsi;
  it.kin = p.d_kin;
  it.Zt = Zt;
  it.Yb = Yb;
  it.V = cur_prec(c) == HPSI_FP64 ? (const void*)p.d_v64 : (const void*)p.d_v32;
  return it;
}

static size_t plane_smem(const Context& c, const Problem& p, int flags) {
  size_t r = 0;
  auto f = [&](auto k) { r = decltype(k)::smem_plane(p, flags & 1, (flags >> 1) & 1); };
  if (cur_prec(c) == HPSI_FP64) dispatch_size<double>(p.n[0], f);
  else dispatch_size<float>(p.n[0], f);
  return r;
}

static int run_batch(Context& c, FastBatch& bt, size_t smem) {
  int rc = HPSI_EINVAL;
  auto go = [&](auto k) { rc = decltype(k)::run(c, bt, smem); };
  if (cur_prec(c) == HPSI_FP64) dispatch_size<double>(bt.N, go);
  else dispatch_size<float>(bt.N, go);
  return rc;
}

static void batch_header(FastBatch& bt, const Problem& p, int flags) {
  bt.nitems = 0;
  bt.N = p.n[0];
  bt.stage_v = flags & 1;
  bt.stage_row = (flags >> 1) & 1;
  bt.tw64 = p.d_ftw64;
  bt.tw32 = p.d_ftw32;
  bt.inv_nr = 1.0 / ((double)p.n[0] * p.n[1] * p.n[2]);
}

// Every plan (staging flags | 4) whose kernels fit the shared memory, for the autotuner.
std::vector<int> local_fast_candidates(const Problem& p, int precision, size_t smem_optin) {
  std::vector<int> out;
  if (p.n[0] != p.n[1] || p.n[1] != p.n[2]) return out;
  auto pick = [&](auto k) {
    using K = decltype(k);
    for (int cand : {3, 2, 1, 0})
      if (K::smem_z() <= smem_optin && K::smem_plane(p, cand & 1, (cand >> 1) & 1) <= smem_optin)
        out.push_back(4 | cand);
  };
  if (precision == HPSI_FP64) dispatch_size<double>(p.n[0], pick);
  else dispatch_size<float>(p.n[0], pick);
  return out;
}

int local_fast_apply(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, void* Zt, void* Yb,
                     int nbb) {
  static FastBatch bt;   // host staging of the parameter block (calls are not thread-safe by contract)
  const int fl = p.fflags[cur_prec(c)];
  batch_header(bt, p, fl);
  const size_t smem = plane_smem(c, p, fl);
  for (int b0 = 0; b0 < nbnd; b0 += nbb) {
    const int nb = std::min(nbb, nbnd - b0);
    bt.nitems = 1;
    bt.item[0] = make_item(c, p, psi + (size_t)b0 * p.npw, hpsi + (size_t)b0 * p.npw, nb, Zt, Yb);
    int rc = run_batch(c, bt, smem);
    if (rc) return rc;
  }
  return HPSI_OK;
}

// Several problems with the same cubic edge and flags in one launch per kernel; scratch[i] holds
// item i's Zt and Y (each n3 * nst * nbnd complex values).
int local_fast_apply_multi(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                           double2* const* hpsi, void* const* zt, void* const* yb) {
  static FastBatch bt;
  int done = 0;
  while (done < nitem) {
    const Problem& p0 = c.probs[prob[done]];
    const int pr = cur_prec(c);
    batch_header(bt, p0, p0.fflags[pr]);
    size_t smem = 0;
    int n = 0;
    while (done + n < nitem && n < kMaxItems) {
      const Problem& p = c.probs[prob[done + n]];
      if (p.n[0] != p0.n[0] || p.fflags[pr] != p0.fflags[pr]) break;
      bt.item[n] = make_item(c, p, psi[done + n], hpsi[done + n], nbnd[done + n], zt[done + n], yb[done + n]);
      smem = std::max(smem, plane_smem(c, p, p.fflags[pr]));
      ++n;
    }
    bt.nitems = n;
    int rc = run_batch(c, bt, smem);
    if (rc) return rc;
    done += n;
  }
  return HPSI_OK;
}

}  // namespace hpsi
