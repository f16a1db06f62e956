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
  int stage_v, stage_row;      // the item's plan: V plane and stick row staged in shared memory
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
  int nitems, N;
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

// Each kernel's work is a tile function of its block coordinates (bx, by, bz), so that the
// persistent batched kernel below runs exactly the same code on the same tiles.
template <typename T, int R1, int R2>
__device__ __forceinline__ void zinv_tile(const FastBatch& bt, int bx, int by, int bz) {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N, G = Gm::G, SC = Gm::GROUPS;
  const FastItem& a = bt.item[bz];
  if (bx * SC >= a.nst || by >= a.nb) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* xbuf = tw + N;                       // [SC][XS]
  V* obuf = xbuf + SC * Gm::XS;           // [N][SC]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * Gm::LPW + lane / G, t = lane % G;
  const bool in_grp = lane < Gm::LPW * G;
  const int s0 = bx * SC, b = by;
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
__global__ void __launch_bounds__(256) k_zinv(const __grid_constant__ FastBatch bt) {
  zinv_tile<T, R1, R2>(bt, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename T, int R1, int R2>
__device__ __forceinline__ void plane_tile(const FastBatch& bt, int bx, int by, int bz) {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N, G = Gm::G, NG = Gm::GROUPS;
  const FastItem& a = bt.item[bz];
  if (by * a.bpc >= a.nb) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  constexpr int PS = Gm::PS;
  V* xbuf = tw + N;                              // [NG][XS]
  V* P = xbuf + NG * Gm::XS;                     // [npl][PS]
  V* row = P + (size_t)a.npl * PS;               // [nst] if stage_row
  T* vpl = reinterpret_cast<T*>(row + (a.stage_row ? a.nst : 0));   // [N][N] if stage_v
  int* xm = reinterpret_cast<int*>(vpl + (a.stage_v ? N * N : 0));  // [N]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * Gm::LPW + lane / G, t = lane % G;
  const bool in_grp = lane < Gm::LPW * G;
  V* xb = xbuf + (in_grp ? grp : 0) * Gm::XS;
  const int j3 = bx;
  const T* Vg = reinterpret_cast<const T*>(a.V) + (size_t)j3 * N * N;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    tw[i] = twt<V>(bt)[i];
    xm[i] = a.xmap[i];
  }
  if (a.stage_v)
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) vpl[i] = Vg[i];
  const T* Vp = a.stage_v ? vpl : Vg;
  for (int bi = 0; bi < a.bpc; ++bi) {
    const int b = by * a.bpc + bi;
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
    V* dst = a.stage_row ? row : yout;
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
    if (a.stage_row) {
      __syncthreads();
      for (int i = threadIdx.x; i < a.nst; i += blockDim.x) yout[i] = row[i];
    }
  }
}

template <typename T, int R1, int R2>
__global__ void __launch_bounds__(256) k_plane(const __grid_constant__ FastBatch bt) {
  plane_tile<T, R1, R2>(bt, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <typename T, int R1, int R2>
__device__ __forceinline__ void zfwd_tile(const FastBatch& bt, int bx, int by, int bz) {
  using V = typename Cx<T>::type;
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N, G = Gm::G, SC = Gm::GROUPS;
  const FastItem& a = bt.item[bz];
  if (bx * SC >= a.nst || by >= a.nb) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw = reinterpret_cast<V*>(smem_raw);
  V* xbuf = tw + N;                       // [SC][XS]
  V* ibuf = xbuf + SC * Gm::XS;           // [N][SC]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp * Gm::LPW + lane / G, t = lane % G;
  const bool in_grp = lane < Gm::LPW * G;
  const int s0 = bx * SC, b = by;
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
__global__ void __launch_bounds__(256) k_zfwd(const __grid_constant__ FastBatch bt) {
  zfwd_tile<T, R1, R2>(bt, blockIdx.x, blockIdx.y, blockIdx.z);
}

#include "nonlocal_tiles.cuh"

// ---- persistent batched H|psi> (hpsi_apply_batch): one cooperative launch over every item ----
// The grid works through the tile list of each phase in turn (the same tile functions as the
// separate kernels: zinv, plane, zfwd, and in float64 the nonlocal calbec, D-scale and add_vuspsi of
// all items), with a grid barrier between phases.  A phase's list holds each item's own tiles only
// (items with fewer bands have fewer), and CTAs take tiles from it one at a time through an atomic
// counter, so that uneven items balance as they do under the hardware block scheduler.  Every wait
// is bounded: on expiry the CTA raises the context's error word and leaves.
struct PersistCtl {
  int nitems;
  int off_z[kMaxItems + 1];   // first zinv / zfwd tile of each item (zch_i x nb_i tiles)
  int off_p[kMaxItems + 1];   // first plane tile of each item (N x ceil(nb_i / bpc) tiles)
  unsigned* bar;              // [0]: arrival counter; [1 + phase]: tile counters; zero at launch
  int* err;
};

constexpr long long kPersistWait = 2000000000LL;   // clock cycles (about 1 s) per barrier wait

__device__ bool persist_sync(unsigned* bar, unsigned target, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    int good = 1;
    const long long t0 = clock64();
    for (unsigned spins = 0;; ++spins) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if ((int)(v - target) >= 0) break;
      if ((spins & 255u) == 255u && (*(volatile int*)err != 0 || clock64() - t0 > kPersistWait)) {
        atomicCAS(err, 0, 3);
        good = 0;
        break;
      }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// The CTA's next tile of a phase (all threads get the same index).
__device__ __forceinline__ int persist_next(unsigned* ctr) {
  __shared__ int tile;
  __syncthreads();   // the previous tile is done with shared memory and with `tile`
  if (threadIdx.x == 0) tile = (int)atomicAdd(ctr, 1u);
  __syncthreads();
  return tile;
}

template <typename T, int R1, int R2, bool NL>
__global__ void __launch_bounds__(256) k_hpsi_batch(const __grid_constant__ FastBatch bt,
                                                    const __grid_constant__ NlBatch nl,
                                                    const __grid_constant__ PersistCtl pc) {
  using Gm = Geo<R1, R2>;
  constexpr int N = Gm::N;
  const unsigned G = gridDim.x;
  const int nz = pc.off_z[pc.nitems], np = pc.off_p[pc.nitems];
  for (int t = persist_next(pc.bar + 1); t < nz; t = persist_next(pc.bar + 1)) {
    const int i = find_item(pc.off_z, pc.nitems, t);
    const int l = t - pc.off_z[i], zch = (bt.item[i].nst + Gm::GROUPS - 1) / Gm::GROUPS;
    zinv_tile<T, R1, R2>(bt, l % zch, l / zch, i);
  }
  if (!persist_sync(pc.bar, G, pc.err)) return;
  for (int t = persist_next(pc.bar + 2); t < np; t = persist_next(pc.bar + 2)) {
    const int i = find_item(pc.off_p, pc.nitems, t);
    const int l = t - pc.off_p[i];
    plane_tile<T, R1, R2>(bt, l % N, l / N, i);
  }
  if (!persist_sync(pc.bar, 2 * G, pc.err)) return;
  for (int t = persist_next(pc.bar + 3); t < nz; t = persist_next(pc.bar + 3)) {
    const int i = find_item(pc.off_z, pc.nitems, t);
    const int l = t - pc.off_z[i], zch = (bt.item[i].nst + Gm::GROUPS - 1) / Gm::GROUPS;
    zfwd_tile<T, R1, R2>(bt, l % zch, l / zch, i);
  }
  if constexpr (NL) {
    // the nonlocal term of every item, added to the local result; its tiles reuse the dynamic
    // shared memory of the FFT phases
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* sm = reinterpret_cast<double2*>(smem_raw);
    if (!persist_sync(pc.bar, 3 * G, pc.err)) return;
    const int nc = nl.off_cal[nl.nitems];
    for (int t = persist_next(pc.bar + 4); t < nc; t = persist_next(pc.bar + 4)) {
      const int i = find_item(nl.off_cal, nl.nitems, t);
      const NlItem& a = nl.item[i];
      const int l = t - nl.off_cal[i], r = l / a.tilesp;
      calbec_tile(a.npw, a.nproj, a.nb, a.kchunk, a.beta, a.psi, a.part, l % a.tilesp, r % a.tilesb, r / a.tilesb,
                  sm);
    }
    if (!persist_sync(pc.bar, 4 * G, pc.err)) return;
    for (int t = blockIdx.x; t < nl.off_ds[nl.nitems]; t += G) {
      const int i = find_item(nl.off_ds, nl.nitems, t);
      const NlItem& a = nl.item[i];
      dscale_one((t - nl.off_ds[i]) * blockDim.x + threadIdx.x, a.nproj, a.nb, a.nsplit, a.part, a.rowptr, a.col,
                 a.dval, a.w);
    }
    if (!persist_sync(pc.bar, 5 * G, pc.err)) return;
    const int na = nl.off_add[nl.nitems];
    for (int t = persist_next(pc.bar + 5); t < na; t = persist_next(pc.bar + 5)) {
      const int i = find_item(nl.off_add, nl.nitems, t);
      const NlItem& a = nl.item[i];
      const int l = t - nl.off_add[i];
      addvus_tile(a.npw, a.nproj, a.nb, a.w, a.beta, a.hpsi, l % a.gtiles, l / a.gtiles, sm);
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
  // Tile grid of the three kernels over the batch; sets each item's bands per k_plane CTA.
  static void geometry(const Context& c, FastBatch& bt, size_t max_plane_smem, int* zch, int* nbmax, int* pyb) {
    int total_rows = 0;
    for (int i = 0; i < bt.nitems; ++i) {
      const FastItem& it = bt.item[i];
      *zch = std::max(*zch, (it.nst + Gm::GROUPS - 1) / Gm::GROUPS);
      *nbmax = std::max(*nbmax, it.nb);
      total_rows += it.nb;
    }
    // bands per k_plane CTA: amortise the staged V plane while keeping >= 2 waves over the batch
    const int occ = max_plane_smem <= c.smem_optin / 2 ? 2 : 1;
    int bpc = std::max(1, (Gm::N * total_rows) / (2 * c.sm_count * occ));
    bpc = std::min(bpc, 8);
    for (int i = 0; i < bt.nitems; ++i) {
      bt.item[i].bpc = bpc;
      *pyb = std::max(*pyb, (bt.item[i].nb + bpc - 1) / bpc);
    }
  }
  // The whole batch in one cooperative launch of k_hpsi_batch (with the float64 nonlocal term when
  // nl is given); *done = false, and nothing launched, when the kernel does not fit.
  static int run_persistent(Context& c, FastBatch& bt, size_t max_plane_smem, const NlBatch* nl, unsigned* bar,
                            bool* done) {
    *done = false;
    const void* kern = nl ? (const void*)k_hpsi_batch<T, R1, R2, true> : (const void*)k_hpsi_batch<T, R1, R2, false>;
    size_t dyn = std::max(smem_z(), max_plane_smem);
    if (nl) dyn = std::max(dyn, sizeof(double2) * (size_t)std::max(CB_SMEM, AV_SMEM));
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess || fa.sharedSizeBytes + dyn > c.smem_optin) {
      cudaGetLastError();
      return HPSI_OK;
    }
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
      cudaGetLastError();
      return HPSI_OK;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, dyn) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      return HPSI_OK;
    }
    static PersistCtl pc;
    int zch = 1, nbmax = 1, pyb = 1;
    geometry(c, bt, max_plane_smem, &zch, &nbmax, &pyb);   // sets each item's bands per plane tile
    pc.nitems = bt.nitems;
    pc.off_z[0] = pc.off_p[0] = 0;
    for (int i = 0; i < bt.nitems; ++i) {
      const FastItem& it = bt.item[i];
      pc.off_z[i + 1] = pc.off_z[i] + ((it.nst + Gm::GROUPS - 1) / Gm::GROUPS) * it.nb;
      pc.off_p[i + 1] = pc.off_p[i] + Gm::N * ((it.nb + it.bpc - 1) / it.bpc);
    }
    pc.bar = bar;
    pc.err = c.d_err;
    static NlBatch empty;   // nitems = 0 (zero-initialised); the float32 form takes no nonlocal phases
    const NlBatch& nb = nl ? *nl : empty;
    cudaError_t e = cudaMemsetAsync(bar, 0, 8 * sizeof(unsigned), c.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "persistent batch barrier reset");
    void* args[] = {(void*)&bt, (void*)&nb, (void*)&pc};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(occ * c.sm_count);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = c.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    HPSI_LAUNCH(c, HPSI_K_BATCH, (e = cudaLaunchKernelExC(&cfg, kern, args)));
    if (e != cudaSuccess) return cuda_fail(c, e, "persistent batched H|psi> launch");
    *done = true;
    return HPSI_OK;
  }
  // One launch of each kernel over every item of the batch (all share the edge N).
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
    int zch = 1, nbmax = 1, pyb = 1;
    geometry(c, bt, max_plane_smem, &zch, &nbmax, &pyb);
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
  const int fl = p.fflags[cur_prec(c)];
  it.stage_v = fl & 1;
  it.stage_row = (fl >> 1) & 1;
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

static void batch_header(FastBatch& bt, const Problem& p) {
  bt.nitems = 0;
  bt.N = p.n[0];
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
  batch_header(bt, p);
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

// Several problems with the same cubic edge in one launch per kernel, each item with its own plan;
// scratch[i] holds item i's Zt and Y (each n3 * nst * nbnd complex values).
int local_fast_apply_multi(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                           double2* const* hpsi, void* const* zt, void* const* yb) {
  static FastBatch bt;
  int done = 0;
  while (done < nitem) {
    const Problem& p0 = c.probs[prob[done]];
    const int pr = cur_prec(c);
    batch_header(bt, p0);
    size_t smem = 0;
    int n = 0;
    while (done + n < nitem && n < kMaxItems) {
      const Problem& p = c.probs[prob[done + n]];
      if (p.n[0] != p0.n[0]) break;
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

// The whole hpsi_apply_batch in one persistent launch: every item on the fast path with one box
// edge, at most kMaxItems of them (and kNlBatch with a nonlocal term in float64).  with_nl:
// the float64 nonlocal term of the items joins the launch.  *done = false: nothing was launched
// and the caller takes the launch-per-kernel path.
int local_batch_persistent(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                           double2* const* hpsi, void* const* zt, void* const* yb, bool with_nl, bool* done) {
  *done = false;
  if (nitem < 1 || nitem > kMaxItems || nitem > kNlBatch || c.force_generic) return HPSI_OK;
  const int pr = cur_prec(c);
  const Problem& p0 = c.probs[prob[0]];
  for (int i = 0; i < nitem; ++i) {
    const Problem& p = c.probs[prob[i]];
    if (!(p.fflags[pr] & 4) || p.n[0] != p0.n[0] || nbnd[i] < 1) return HPSI_OK;
  }
  static FastBatch bt;
  static NlBatch nl;
  batch_header(bt, p0);
  size_t smem = 0;
  for (int i = 0; i < nitem; ++i) {
    const Problem& p = c.probs[prob[i]];
    bt.item[i] = make_item(c, p, psi[i], hpsi[i], nbnd[i], zt[i], yb[i]);
    smem = std::max(smem, plane_smem(c, p, p.fflags[pr]));
  }
  bt.nitems = nitem;
  const NlBatch* nlp = nullptr;
  if (with_nl) {
    // partial sums and w of every item side by side in the workspace (as the launch-per-kernel form)
    std::vector<size_t> off(nitem);
    std::vector<int> ns(nitem), kc(nitem);
    size_t total = 0;
    for (int i = 0; i < nitem; ++i) {
      size_t bytes = 0;
      nonlocal_fp64_plan(c, c.probs[prob[i]], nbnd[i], &ns[i], &kc[i], &bytes);
      off[i] = total;
      total += (bytes + 255) & ~size_t(255);
    }
    int rc = ensure_buffer(c, &c.ws.part, &c.ws.partbytes, std::max<size_t>(total, 256));
    if (rc) return rc;
    unsigned char* base = static_cast<unsigned char*>(c.ws.part);
    int n = 0;
    nl.off_cal[0] = nl.off_ds[0] = nl.off_add[0] = 0;
    for (int i = 0; i < nitem; ++i) {
      const Problem& p = c.probs[prob[i]];
      if (p.nproj == 0) continue;
      NlItem& a = nl.item[n];
      a.npw = p.npw;
      a.nproj = p.nproj;
      a.nb = nbnd[i];
      a.kchunk = kc[i];
      a.nsplit = ns[i];
      a.tp = CB_TP;
      a.tilesp = (p.nproj + CB_TP - 1) / CB_TP;
      a.tilesb = (a.nb + CB_TB - 1) / CB_TB;
      a.gtiles = (p.npw + AV_TG - 1) / AV_TG;
      a.beta = p.d_beta;
      a.psi = psi[i];
      a.hpsi = hpsi[i];
      a.part = reinterpret_cast<double2*>(base + off[i]);
      a.w = a.part + (size_t)a.nsplit * a.nb * a.nproj;
      a.rowptr = p.d_rowptr;
      a.col = p.d_col;
      a.dval = p.d_dval;
      nl.off_cal[n + 1] = nl.off_cal[n] + a.tilesp * a.tilesb * a.nsplit;
      nl.off_ds[n + 1] = nl.off_ds[n] + (a.nproj * a.nb + 255) / 256;
      nl.off_add[n + 1] = nl.off_add[n] + a.gtiles * ((a.nb + AV_TB - 1) / AV_TB);
      ++n;
    }
    nl.nitems = n;
    if (n > 0) nlp = &nl;
  }
  int rc = ensure_buffer(c, &c.ws.pbar, &c.ws.pbarbytes, 256);
  if (rc) return rc;
  unsigned* bar = static_cast<unsigned*>(c.ws.pbar);
  rc = HPSI_EINVAL;
  auto go = [&](auto k) { rc = decltype(k)::run_persistent(c, bt, smem, nlp, bar, done); };
  if (pr == HPSI_FP64) dispatch_size<double>(bt.N, go);
  else dispatch_size<float>(bt.N, go);
  return rc;
}

}  // namespace hpsi
