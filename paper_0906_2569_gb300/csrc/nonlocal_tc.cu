// Nonlocal contractions of the mixed-precision path on the 5th-generation tensor cores.
//
// Separable projectors (paper Sec. 3): becp = <beta|psi>, w = D becp, hpsi += beta w.  Both
// contractions are dense and run as real bf16 GEMMs with float32 accumulation in TMEM:
//
//   complex -> real:  with psi, beta, w stored as interleaved (re, im) real rows,
//     calbec      C[p][n] = sum_k A[p][k] B[n][k],  A = beta (K = 2 npw),
//                 B rows n < nb: psi_n (re, im); rows nb + b: (im, -re) of psi_b
//                 -> C[p][b] = Re<beta_p|psi_b>, C[p][nb+b] = Im<beta_p|psi_b>
//     add_vuspsi  C[b][n] = sum_k A[b][k] B[n][k],  A = w (K = 2P), B[2G+c][2p+c'] built from
//                 beta so that C[b][2G] = Re(sum_p w_bp beta_p(G)), C[b][2G+1] = Im(...)
//   precision:  every float64 operand x is split into bf16 terms x = x0 + x1 (+ x2) and the
//     products x_i y_j with i + j < NT are accumulated (NT = 2: three products, ~16 significant
//     bits; NT = 3: six products).
//
// Kernel: one CTA (4 warps) per 128 x 128 output tile (and per K-split for calbec).  Warp 0 lane 0
// streams 128x64 bf16 tiles with TMA (128-byte swizzle) through a multi-stage mbarrier ring;
// warp 1 lane 0 issues tcgen05.mma (M = 128, N = 128, K = 16) into one TMEM accumulator of 128
// columns; all four warps read the accumulator back with tcgen05.ld (one TMEM lane per thread) and
// write the epilogue.  Every wait is bounded by a clock limit: on expiry the CTA raises the
// context's error word, drains what it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "hpsi_internal.h"

namespace hpsi {

namespace {

constexpr int TBM = 128;             // rows of A per tile (TMEM lanes)
constexpr int TBN = 128;             // rows of B per tile (accumulator columns)
constexpr int TBK = 64;              // bf16 per 128-byte swizzled row
constexpr int kTileBytes = TBM * TBK * 2;   // 16 KB, A and B tiles alike
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr int kInnerKsteps = 8;      // subspace inner products: K steps per float32 accumulation
constexpr int kCalbecKsteps = 16;    // calbec: at most this many K steps per float32 accumulation by default;
                                     // the error of a float32 accumulation grows with its length, and
                                     // the partial sums of the splits are added in float64
constexpr int kAddKsteps = 8;        // add_vuspsi: at most this many K steps (of K = 2P) per float32
                                     // accumulation; more splits are added in float64 (the measured
                                     // error of one long accumulation grows in proportion to P)

template <int NT> struct TcCfg {
  static constexpr int stages = NT == 2 ? 3 : 2;
  static constexpr int stage_bytes = 2 * NT * kTileBytes;
  static constexpr int smem = stages * stage_bytes + 1024;
};

struct TcArgs {
  int M, N;          // logical rows of A and of B (output is M x N)
  int nksteps;       // K / 64
  int ksplit;        // K-steps per split (gridDim.z splits)
  int mode;          // 0: store float partials [split][M][N]; 1: add into complex128 rows
  float* part;
  double2* out;      // mode 1: out[m][n/2] += (C[m][n], C[m][n+1]) for even n
  int ldo;           // mode 1: complex elements per output row
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false if the clock limit expired or another thread of the CTA aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          long long limit = kWaitCycles) {
  const long long t0 = clock64();
  for (unsigned it = 0;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort_flag) return false;
      if (clock64() - t0 > limit) {
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// Self-test of the failure path: one thread waits, with a short limit, on an mbarrier that no
// thread and no copy ever arrives at; the expiry raises the error word exactly as in k_tc_gemm.
__global__ void k_wait_selftest(int* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ volatile int abort_flag;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
    if (!mbar_wait(smem_u32(&bar), 0, &abort_flag, limit)) atomicExch(err, 1);
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// K-major operand, 128-byte swizzle: 8-row groups of 128-byte rows, 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;              // leading byte offset (not used by swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// kind::f16 instruction descriptor: D f32, A and B bf16, both K-major, M = 128, N = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) |
                            ((uint32_t)(TBM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
               : "memory");
}

template <int NT>
__global__ void __launch_bounds__(128, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
              const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tB0,
              const __grid_constant__ CUtensorMap tB1, const __grid_constant__ CUtensorMap tB2, TcArgs a) {
  using Cfg = TcCfg<NT>;
  constexpr int S = Cfg::stages;
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  __shared__ __align__(8) uint64_t full_bar[S];
  __shared__ __align__(8) uint64_t empty_bar[S];
  __shared__ __align__(8) uint64_t acc_bar;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile_n = blockIdx.x * TBN, tile_m = blockIdx.y * TBM, split = blockIdx.z;
  const int kbeg = split * a.ksplit, kend = min(a.nksteps, kbeg + a.ksplit);
  const int nk = kend - kbeg;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty_bar[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&acc_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_flag = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(TBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  const CUtensorMap* mA[3] = {&tA0, &tA1, &tA2};
  const CUtensorMap* mB[3] = {&tB0, &tB1, &tB2};

  int issued[S];
#pragma unroll
  for (int s = 0; s < S; ++s) issued[s] = 0;
  if (warp == 0 && lane == 0 && nk > 0) {
    // producer
    for (int i = 0; i < nk; ++i) {
      const int s = i % S, round = i / S;
      if (round > 0 && !mbar_wait(smem_u32(&empty_bar[s]), (round - 1) & 1, &abort_flag)) break;
      const uint32_t fb = smem_u32(&full_bar[s]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(Cfg::stage_bytes)
                   : "memory");
      unsigned char* st = smem + s * Cfg::stage_bytes;
      const int kx = (kbeg + i) * TBK;
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        tma_load_2d(smem_u32(st + t * kTileBytes), mA[t], kx, tile_m, fb);
        tma_load_2d(smem_u32(st + (NT + t) * kTileBytes), mB[t], kx, tile_n, fb);
      }
      issued[s] = round + 1;
    }
  } else if (warp == 1 && lane == 0 && nk > 0) {
    // MMA issuer
    uint32_t acc = 0;
    for (int i = 0; i < nk; ++i) {
      const int s = i % S, round = i / S;
      if (!mbar_wait(smem_u32(&full_bar[s]), round & 1, &abort_flag)) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const unsigned char* st = smem + s * Cfg::stage_bytes;
      // smallest products first: the float32 accumulation rounds (with a bias, measured) relative to
      // the running sum, so the 2^-16 and 2^-8 terms go in while it is still small and only the last
      // four MMAs of a K-step, the leading products, round at full magnitude
#pragma unroll
      for (int lvl = NT - 1; lvl >= 0; --lvl)
#pragma unroll
        for (int ia = 0; ia <= lvl; ++ia) {
          const int ib = lvl - ia;
#pragma unroll
          for (int kk = 0; kk < TBK / 16; ++kk) {
            const uint64_t da = sw128_desc(smem_u32(st + ia * kTileBytes) + kk * 32);
            const uint64_t db = sw128_desc(smem_u32(st + (NT + ib) * kTileBytes) + kk * 32);
            mma_bf16(tmem, da, db, acc);
            acc = 1;
          }
        }
      mma_commit(smem_u32(&empty_bar[s]));
    }
    mma_commit(smem_u32(&acc_bar));
  }
  __syncwarp();
  // epilogue: wait for the accumulator, TMEM lane = output row
  bool ok = nk > 0 && mbar_wait(smem_u32(&acc_bar), 0, &abort_flag);
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (ok && !abort_flag) {
    const int row = tile_m + warp * 32 + lane;
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < TBN; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(lane_addr + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (row < a.M) {
        const int n0 = tile_n + c0;
        if (a.mode == 0) {
          float* o = a.part + ((size_t)split * a.M + row) * a.N;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (n0 + j < a.N) o[n0 + j] = __uint_as_float(r[j]);
        } else {
          double2* o = a.out + (size_t)row * a.ldo + (n0 >> 1);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (n0 + 2 * j < a.N) {
              double2 v = o[j];
              v.x += (double)__uint_as_float(r[2 * j]);
              v.y += (double)__uint_as_float(r[2 * j + 1]);
              o[j] = v;
            }
        }
      }
    }
  }
  if (abort_flag && threadIdx.x == 0) atomicExch(a.err, 1);
  // drain: every TMA this CTA issued has landed before the CTA (and its shared memory) goes away
  if (warp == 0 && lane == 0) {
    volatile int never = 0;
    for (int s = 0; s < S; ++s)
      if (issued[s] > 0) mbar_wait(smem_u32(&full_bar[s]), (issued[s] - 1) & 1, &never);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TBN));
}

// hpsi[b][g] += sum_s (part[s][b][2g], part[s][b][2g+1]), summed in float64
__global__ void k_add_partials(int nb, int npw, int nsplit, const float* __restrict__ part, double2* __restrict__ hpsi) {
  const size_t n = (size_t)nb * npw, plane = 2 * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float2* p = reinterpret_cast<const float2*>(part) + i;
    double sx = 0.0, sy = 0.0;
    for (int s = 0; s < nsplit; ++s) {
      const float2 v = p[(size_t)s * (plane / 2)];
      sx += (double)v.x;
      sy += (double)v.y;
    }
    double2 o = hpsi[i];
    o.x += sx;
    o.y += sy;
    hpsi[i] = o;
  }
}

// ---- operand preparation ----------------------------------------------------------------------

template <int NT>
__device__ __forceinline__ void split_store(double x, __nv_bfloat16* p0, size_t plane, size_t idx) {
  double r = x;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)r);
    p0[t * plane + idx] = h;
    r -= (double)__bfloat162float(h);
  }
}

// A of calbec: row p = beta_p as (re, im) pairs, K padded with zeros to kc.
template <int NT>
__global__ void k_split_beta_cal(int nproj, int npw, int kc, const double2* __restrict__ beta,
                                 __nv_bfloat16* __restrict__ out) {
  const size_t plane = (size_t)nproj * kc;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(i / kc), k = (int)(i % kc);
    double x = 0.0;
    if (k < 2 * npw) {
      const double2 v = beta[(size_t)p * npw + (k >> 1)];
      x = (k & 1) ? v.y : v.x;
    }
    split_store<NT>(x, out, plane, i);
  }
}

// B of add_vuspsi: row n = 2G + c, column k = 2p + c':  c=0: (re, -im), c=1: (im, re) of beta_p(G).
template <int NT>
__global__ void k_split_beta_add(int nproj, int npw, int ka, const double2* __restrict__ beta,
                                 __nv_bfloat16* __restrict__ out) {
  const size_t plane = (size_t)2 * npw * ka;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(i / ka), k = (int)(i % ka);
    double x = 0.0;
    if (k < 2 * nproj) {
      const double2 v = beta[(size_t)(k >> 1) * npw + (n >> 1)];
      const int c = n & 1, cp = k & 1;
      x = c == 0 ? (cp == 0 ? v.x : -v.y) : (cp == 0 ? v.y : v.x);
    }
    split_store<NT>(x, out, plane, i);
  }
}

// B of calbec: rows b < nb: psi_b (re, im); rows nb + b: (im, -re).  One thread per complex psi
// element (or per pair of padding columns), writing bf16 pairs.
template <int NT>
__global__ void k_split_psi(int nb, int npw, int kc, const double2* __restrict__ psi, __nv_bfloat16* __restrict__ out) {
  const size_t plane = (size_t)2 * nb * kc;
  const int half = kc / 2;   // complex columns including the zero padding
  const size_t n = (size_t)nb * half;
  __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(out);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / half), g = (int)(i - (size_t)b * half);
    double2 v = make_double2(0.0, 0.0);
    if (g < npw) v = psi[(size_t)b * npw + g];
    double r0 = v.x, r1 = v.y;      // row b:      (re, im)
    double s0 = v.y, s1 = -v.x;     // row nb + b: (im, -re)
    const size_t i0 = ((size_t)b * kc) / 2 + g, i1 = ((size_t)(nb + b) * kc) / 2 + g;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn((float)r0), h1 = __float2bfloat16_rn((float)r1);
      const __nv_bfloat16 k0 = __float2bfloat16_rn((float)s0), k1 = __float2bfloat16_rn((float)s1);
      o2[t * (plane / 2) + i0] = __halves2bfloat162(h0, h1);
      o2[t * (plane / 2) + i1] = __halves2bfloat162(k0, k1);
      r0 -= (double)__bfloat162float(h0);
      r1 -= (double)__bfloat162float(h1);
      s0 -= (double)__bfloat162float(k0);
      s1 -= (double)__bfloat162float(k1);
    }
  }
}

// out[i] = sum over the K-splits s of part[s][i] (float64, splits in order), i < n: the partials
// of calbec summed once, so that the D-scale reads each <beta_q|psi_b> once per use instead of
// re-adding its nsplit partials for every nonzero D_pq
__global__ void k_sum_partials(size_t n, int nsplit, const float* __restrict__ part, double* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
#pragma unroll 8
    for (int k = 0; k < nsplit; ++k) s += (double)part[(size_t)k * n + i];
    out[i] = s;
  }
}

// w[b][p] = sum_q D_pq becp[b][q], becp from the partials [split][P][2 nb] (float, summed in
// float64, or already summed: S = double, nsplit = 1); written as the bf16 terms of A of
// add_vuspsi, row b = (re, im) pairs of w_b.
template <int NT, typename S>
__global__ void k_dscale_tc(int nproj, int nb, int nsplit, int ka, const S* __restrict__ part,
                            const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double2* __restrict__ val, __nv_bfloat16* __restrict__ wa) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nproj * nb) return;
  const int b = i / nproj, p = i % nproj;
  const int N = 2 * nb;
  double wr = 0.0, wi = 0.0;
  for (int e = rowptr[p]; e < rowptr[p + 1]; ++e) {
    const int q = col[e];
    double sr = 0.0, si = 0.0;
    for (int s = 0; s < nsplit; ++s) {
      const S* ps = part + ((size_t)s * nproj + q) * N;
      sr += (double)ps[b];
      si += (double)ps[nb + b];
    }
    const double2 d = val[e];
    wr += d.x * sr - d.y * si;
    wi += d.x * si + d.y * sr;
  }
  const size_t plane = (size_t)nb * ka;
  split_store<NT>(wr, wa, plane, (size_t)b * ka + 2 * p);
  split_store<NT>(wi, wa, plane, (size_t)b * ka + 2 * p + 1);
}

// Rows r0 .. r1-1 of a complex64 block [rows][npw] as (re, im) bf16 pairs, K padded with zeros to
// kc, into NT term planes of plane elements each (A of the subspace inner products).  One thread per
// complex element or padding pair.
template <int NT>
__global__ void k_split_rows32(int r0, int r1, int npw, int kc, size_t plane, const float2* __restrict__ src,
                               __nv_bfloat16* __restrict__ out) {
  const int half = kc / 2;
  const size_t n = (size_t)(r1 - r0) * half;
  __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(out);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int row = r0 + (int)(i / half), g = (int)(i % half);
    float2 v = make_float2(0.f, 0.f);
    if (g < npw) v = src[(size_t)row * npw + g];
    float x = v.x, y = v.y;
    const size_t at = ((size_t)row * kc) / 2 + g;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const __nv_bfloat16 hx = __float2bfloat16_rn(x), hy = __float2bfloat16_rn(y);
      o2[t * (plane / 2) + at] = __halves2bfloat162(hx, hy);
      x -= __bfloat162float(hx);   // exact: the remainder of a float32 after a bf16 rounding
      y -= __bfloat162float(hy);
    }
  }
}

// B of the subspace inner products from a complex64 block [nb][npw]: rows b: (re, im); rows nb + b:
// (im, -re), K padded to kc (the calbec form, so that C[i][b] = Re<a_i|x_b>, C[i][nb+b] = Im).
template <int NT>
__global__ void k_split_inner_b(int nb, int npw, int kc, const float2* __restrict__ src,
                                __nv_bfloat16* __restrict__ out) {
  const size_t plane = (size_t)2 * nb * kc;
  const int half = kc / 2;
  const size_t n = (size_t)nb * half;
  __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(out);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(i / half), g = (int)(i % half);
    float2 v = make_float2(0.f, 0.f);
    if (g < npw) v = src[(size_t)b * npw + g];
    float r0 = v.x, r1 = v.y, s0 = v.y, s1 = -v.x;
    const size_t i0 = ((size_t)b * kc) / 2 + g, i1 = ((size_t)(nb + b) * kc) / 2 + g;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn(r0), h1 = __float2bfloat16_rn(r1);
      const __nv_bfloat16 k0 = __float2bfloat16_rn(s0), k1 = __float2bfloat16_rn(s1);
      o2[t * (plane / 2) + i0] = __halves2bfloat162(h0, h1);
      o2[t * (plane / 2) + i1] = __halves2bfloat162(k0, k1);
      r0 -= __bfloat162float(h0);
      r1 -= __bfloat162float(h1);
      s0 -= __bfloat162float(k0);
      s1 -= __bfloat162float(k1);
    }
  }
}

// out[i + b ldo] = (sum_s part[s][i][b], sum_s part[s][i][nb + b]), summed in float64; part is
// [nsplit][M][2 nb].  Threads run over b fastest (coalesced partial reads).
__global__ void k_inner_reduce(int M, int nb, int nsplit, const float* __restrict__ part, double2* __restrict__ out64,
                               float2* __restrict__ out32, int ldo) {
  const size_t n = (size_t)M * nb, N = (size_t)2 * nb;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(t % nb), i = (int)(t / nb);
    double re = 0.0, im = 0.0;
    for (int s = 0; s < nsplit; ++s) {
      const float* ps = part + ((size_t)s * M + i) * N;
      re += (double)ps[b];
      im += (double)ps[nb + b];
    }
    if (out64) out64[(size_t)b * ldo + i] = make_double2(re, im);
    else out32[(size_t)b * ldo + i] = make_float2((float)re, (float)im);
  }
}

// ---- Gamma-point real form: operands ------------------------------------------------------------

// B of add_vuspsi in the real form: row r (real-basis coordinate), column k = projector (K padded
// to ka): betar[k][r].  Setup only.
template <int NT>
__global__ void k_split_betar_add(int nproj, int nr, int ka, const double* __restrict__ betar,
                                  __nv_bfloat16* __restrict__ out) {
  const size_t plane = (size_t)nr * ka;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / ka), k = (int)(i % ka);
    split_store<NT>(k < nproj ? betar[(size_t)k * nr + r] : 0.0, out, plane, i);
  }
}

// B of calbec in the real form: row b = x_b (nr real coordinates, K padded to kc with zeros);
// scaled = 0: x holds coefficients and r >= 2 is multiplied by sqrt2.  One thread per pair of
// coordinates, band b = blockIdx.y.
template <int NT, typename R>
__global__ void k_split_xr(int nb, int nr, int kc, int scaled, const R* __restrict__ x,
                           __nv_bfloat16* __restrict__ out) {
  const size_t plane = (size_t)nb * kc;
  const int half = kc / 2, b = blockIdx.y;
  __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(out);
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < half; h += gridDim.x * blockDim.x) {
    const size_t at = (size_t)b * half + h;
    if constexpr (sizeof(R) == 4) {
      // float32 input: the three bf16 terms of a float are exact, and float32 arithmetic finds them
      float r0 = 0.f, r1 = 0.f;
      if (2 * h < nr) {
        const float2 v = *reinterpret_cast<const float2*>(x + (size_t)b * nr + 2 * h);
        r0 = v.x;
        r1 = v.y;
        if (!scaled && h > 0) {
          r0 *= 1.41421356f;
          r1 *= 1.41421356f;
        }
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(r0), h1 = __float2bfloat16_rn(r1);
        o2[t * (plane / 2) + at] = __halves2bfloat162(h0, h1);
        r0 -= __bfloat162float(h0);
        r1 -= __bfloat162float(h1);
      }
    } else {
      double r0 = 0.0, r1 = 0.0;
      if (2 * h < nr) {
        r0 = (double)x[(size_t)b * nr + 2 * h];
        r1 = (double)x[(size_t)b * nr + 2 * h + 1];
        if (!scaled && h > 0) {
          r0 *= 1.4142135623730950488;
          r1 *= 1.4142135623730950488;
        }
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn((float)r0), h1 = __float2bfloat16_rn((float)r1);
        o2[t * (plane / 2) + at] = __halves2bfloat162(h0, h1);
        r0 -= (double)__bfloat162float(h0);
        r1 -= (double)__bfloat162float(h1);
      }
    }
  }
}

// w[b][p] = sum_q D'_pq becp[q][b] with becp from the partials [split][P][nb] (float, summed in
// float64, or already summed: S = double, nsplit = 1), written as the bf16 terms of A of the real
// add_vuspsi (row b, K = projector, pad ka).
template <int NT, typename S>
__global__ void k_dscale_tc_r(int nproj, int nb, int nsplit, int ka, const S* __restrict__ part,
                              const int* __restrict__ rowptr, const int* __restrict__ col,
                              const double* __restrict__ val, __nv_bfloat16* __restrict__ wa) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nproj * nb) return;
  const int b = i / nproj, p = i % nproj;
  double acc = 0.0;
  for (int e = rowptr[p]; e < rowptr[p + 1]; ++e) {
    const int q = col[e];
    double sq = 0.0;
    for (int s = 0; s < nsplit; ++s) sq += (double)part[((size_t)s * nproj + q) * nb + b];
    acc = fma(val[e], sq, acc);
  }
  split_store<NT>(acc, wa, (size_t)nb * ka, (size_t)b * ka + p);
}

// A of add_vuspsi from float64 rows: out[row][k] = src[row][k] for k < kin, 0 up to kpad (w as
// interleaved (re, im) pairs, kin = 2P, or real, kin = P).
template <int NT>
__global__ void k_split_rows64(int rows, int kin, int kpad, const double* __restrict__ src,
                               __nv_bfloat16* __restrict__ out) {
  const size_t plane = (size_t)rows * kpad;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < plane; i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / kpad), k = (int)(i % kpad);
    split_store<NT>(k < kin ? src[(size_t)r * kin + k] : 0.0, out, plane, i);
  }
}

// ---- host side ------------------------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int get_encoder(Context& c) {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  });
  if (!g_encode) return fail(c, HPSI_ECUDA, "cuTensorMapEncodeTiled is not available");
  return HPSI_OK;
}

// Map over a K-major bf16 matrix [rows][kpad], tiles of 128 rows x 64 columns, 128-byte swizzle.
int make_map(Context& c, CUtensorMap* m, const void* base, int rows, int kpad) {
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (kpad % TBK)) return fail(c, HPSI_EINVAL, "tensor map alignment");
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)TBM};
  cuuint32_t es[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(c, HPSI_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return HPSI_OK;
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// pa_stride / pb_stride: elements between the bf16 term planes of A / B (0: rows x kpad, packed)
template <int NT>
int launch_gemm(Context& c, const void* A, int M, const void* B, int N, int kpad, int nsplit, int ksplit, int mode,
                float* part, double2* out, int ldo, int kernel_class, size_t pa_stride = 0, size_t pb_stride = 0) {
  CUtensorMap ma[3], mb[3];
  const size_t pa = pa_stride ? pa_stride : (size_t)M * kpad, pb = pb_stride ? pb_stride : (size_t)N * kpad;
  for (int t = 0; t < 3; ++t) {
    const int tt = t < NT ? t : NT - 1;
    int rc = make_map(c, &ma[t], static_cast<const __nv_bfloat16*>(A) + tt * pa, M, kpad);
    if (rc) return rc;
    rc = make_map(c, &mb[t], static_cast<const __nv_bfloat16*>(B) + tt * pb, N, kpad);
    if (rc) return rc;
  }
  TcArgs a;
  a.M = M;
  a.N = N;
  a.nksteps = kpad / TBK;
  a.ksplit = ksplit;
  a.mode = mode;
  a.part = part;
  a.out = out;
  a.ldo = ldo;
  a.err = c.d_err;
  static bool attr[4] = {false, false, false, false};
  if (!attr[NT]) {
    cudaFuncSetAttribute(k_tc_gemm<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<NT>::smem);
    attr[NT] = true;
  }
  dim3 grid((N + TBN - 1) / TBN, (M + TBM - 1) / TBM, nsplit);
  HPSI_LAUNCH(c, kernel_class,
              (k_tc_gemm<NT><<<grid, 128, TcCfg<NT>::smem, c.stream>>>(ma[0], ma[1], ma[2], mb[0], mb[1], mb[2], a)));
  return HPSI_OK;
}

template <int NT>
int prepare_t(Context& c, Problem& p) {
  const int P = p.nproj, npw = p.npw;
  const int kc = round_up(2 * npw, TBK), ka = round_up(2 * P, TBK);
  const size_t cal = (size_t)NT * P * kc, add = (size_t)NT * 2 * npw * ka;
  cudaError_t e = cudaMalloc((void**)&p.d_beta_bf, sizeof(__nv_bfloat16) * (cal + add));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HPSI_ENOMEM, "device allocation of the bf16 projector terms failed");
  }
  __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(p.d_beta_bf);
  HPSI_LAUNCH(c, HPSI_K_SPLIT, (k_split_beta_cal<NT><<<4 * c.sm_count, 256, 0, c.stream>>>(P, npw, kc, p.d_beta, base)));
  HPSI_LAUNCH(c, HPSI_K_SPLIT,
              (k_split_beta_add<NT><<<4 * c.sm_count, 256, 0, c.stream>>>(P, npw, ka, p.d_beta, base + cal)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "bf16 projector split");
  return HPSI_OK;
}

template <int NT>
int apply_t(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, int kmax);

// Autotuner of the mixed calbec's K-split: on the first application of a problem with >= 4 bands
// (not under stream capture), time the caps of 4, 8 and 16 K-steps per float32 accumulation on
// this call's own bands (one warm-up and one timed run each) and keep the fastest.  Every
// candidate is at or below the default cap, so none is less accurate than the default.
template <int NT>
int tune_ksplit(Context& c, const Problem& p, const double2* psi, int nbnd) {
  // add_vuspsi adds into its output, so the timed runs write a scratch block, not the caller's
  cudaEvent_t e0, e1;
  double2* scratch = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMalloc((void**)&scratch, sizeof(double2) * (size_t)nbnd * p.npw) != cudaSuccess) {
    cudaGetLastError();
    p.nl_kmax = kCalbecKsteps;
    return HPSI_OK;
  }
  double2* hpsi = scratch;
  const bool timing = c.timing;
  c.timing = false;
  float best = 1e30f;
  int pick = kCalbecKsteps, rc = HPSI_OK;
  for (int km : {kCalbecKsteps, 8, 4}) {
    float ms = 0.f;
    for (int rep = 0; rep < 2 && !rc; ++rep) {
      cudaEventRecord(e0, c.stream);
      rc = apply_t<NT>(c, p, psi, hpsi, nbnd, km);
      cudaEventRecord(e1, c.stream);
    }
    if (rc) break;
    if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) {
      best = ms;
      pick = km;
    }
  }
  c.timing = timing;
  cudaStreamSynchronize(c.stream);
  cudaFree(scratch);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p.nl_kmax = pick;
  return rc;
}

template <int NT>
int apply_t(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, int kmax) {
  const int P = p.nproj, npw = p.npw;
  const int kc = round_up(2 * npw, TBK), ka = round_up(2 * P, TBK);
  const size_t cal = (size_t)NT * P * kc;
  const __nv_bfloat16* bcal = reinterpret_cast<const __nv_bfloat16*>(p.d_beta_bf);
  const __nv_bfloat16* badd = bcal + cal;
  // split-K of calbec: about two CTAs per SM over all output tiles
  const int nks = kc / TBK;
  const int tiles = ((2 * nbnd + TBN - 1) / TBN) * ((P + TBM - 1) / TBM);
  int nsplit = std::max(1, std::min(nks, (2 * c.sm_count + tiles - 1) / tiles));
  int ksplit = (nks + nsplit - 1) / nsplit;
  ksplit = std::min(ksplit, kmax);
  nsplit = (nks + ksplit - 1) / ksplit;
  const size_t psib = sizeof(__nv_bfloat16) * (size_t)NT * 2 * nbnd * kc;
  const size_t partb = sizeof(float) * (size_t)nsplit * P * 2 * nbnd;
  const size_t wab = sizeof(__nv_bfloat16) * (size_t)NT * nbnd * ka;
  // add_vuspsi in K-splits of at most kAddKsteps steps when 2P is longer than that
  const int naks = ka / TBK;
  const int aksplit = (naks + (naks + kAddKsteps - 1) / kAddKsteps - 1) / ((naks + kAddKsteps - 1) / kAddKsteps);
  const int ansplit = (naks + aksplit - 1) / aksplit;   // every split has at least one K step
  const size_t addb = ansplit > 1 ? sizeof(float) * (size_t)ansplit * nbnd * 2 * npw : 0;
  const size_t becb = nsplit > 1 ? sizeof(double) * (size_t)P * 2 * nbnd : 0;
  const size_t need = psib + partb + wab + addb + becb + 5 * 256;
  int rc = ensure_buffer(c, &c.ws.mixed, &c.ws.mixedbytes, need);
  if (rc) return rc;
  unsigned char* w0 = static_cast<unsigned char*>(c.ws.mixed);
  __nv_bfloat16* psi_bf = reinterpret_cast<__nv_bfloat16*>(w0);
  float* part = reinterpret_cast<float*>(w0 + ((psib + 255) & ~size_t(255)));
  __nv_bfloat16* wa =
      reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(part) + ((partb + 255) & ~size_t(255)));
  // the K padding of w (columns 2P .. ka) is not written by the D-scale kernel
  cudaError_t e0 = cudaMemsetAsync(wa, 0, wab, c.stream);
  if (e0 != cudaSuccess) return cuda_fail(c, e0, "workspace clear");
  const int split_grid = (int)std::min<size_t>(8 * c.sm_count, ((size_t)nbnd * (kc / 2) + 255) / 256);
  HPSI_LAUNCH(c, HPSI_K_SPLIT, (k_split_psi<NT><<<split_grid, 256, 0, c.stream>>>(nbnd, npw, kc, psi, psi_bf)));
  rc = launch_gemm<NT>(c, bcal, P, psi_bf, 2 * nbnd, kc, nsplit, ksplit, 0, part, nullptr, 0, HPSI_K_CALBEC);
  if (rc) return rc;
  const int n = P * nbnd;
  float* apart = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(wa) + ((wab + 255) & ~size_t(255)));
  if (nsplit > 1) {
    double* becp = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(apart) + ((addb + 255) & ~size_t(255)));
    const size_t nel = (size_t)P * 2 * nbnd;
    HPSI_LAUNCH(c, HPSI_K_DSCALE, (k_sum_partials<<<(int)std::min<size_t>(8 * c.sm_count, (nel + 255) / 256), 256, 0,
                                                    c.stream>>>(nel, nsplit, part, becp)));
    HPSI_LAUNCH(c, HPSI_K_DSCALE,
                (k_dscale_tc<NT, double><<<(n + 255) / 256, 256, 0, c.stream>>>(P, nbnd, 1, ka, becp, p.d_rowptr,
                                                                                p.d_col, p.d_dval, wa)));
  } else {
    HPSI_LAUNCH(c, HPSI_K_DSCALE,
                (k_dscale_tc<NT, float><<<(n + 255) / 256, 256, 0, c.stream>>>(P, nbnd, 1, ka, part, p.d_rowptr,
                                                                               p.d_col, p.d_dval, wa)));
  }
  if (ansplit > 1) {
    rc = launch_gemm<NT>(c, wa, nbnd, badd, 2 * npw, ka, ansplit, aksplit, 0, apart, nullptr, 0, HPSI_K_ADDVUS);
    if (rc) return rc;
    const size_t nel = (size_t)nbnd * npw;
    HPSI_LAUNCH(c, HPSI_K_ADDVUS, (k_add_partials<<<(int)std::min<size_t>(8 * c.sm_count, (nel + 255) / 256), 256, 0,
                                                    c.stream>>>(nbnd, npw, ansplit, apart, hpsi)));
  } else {
    rc = launch_gemm<NT>(c, wa, nbnd, badd, 2 * npw, ka, 1, naks, 1, nullptr, hpsi, npw, HPSI_K_ADDVUS);
    if (rc) return rc;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core nonlocal kernels launch");
  return HPSI_OK;
}

template <int NT>
int gamma_prepare_t(Context& c, Problem& p) {
  const int P = p.nproj, nh = (p.npw + 1) / 2, nr = 2 * nh;
  const int kc = round_up(nr, TBK), ka = round_up(P, TBK);
  const size_t cal = (size_t)NT * P * kc, add = (size_t)NT * nr * ka;
  cudaError_t e = cudaMalloc((void**)&p.d_betar_bf, sizeof(__nv_bfloat16) * (cal + add));
  if (e != cudaSuccess) {
    cudaGetLastError();
    p.d_betar_bf = nullptr;
    return fail(c, HPSI_ENOMEM, "device allocation of the Gamma-form bf16 projector terms failed");
  }
  __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(p.d_betar_bf);
  // calbec's A: the rows of betar read as interleaved pairs (nh pairs of a 2 nh row)
  HPSI_LAUNCH(c, HPSI_K_SPLIT, (k_split_beta_cal<NT><<<4 * c.sm_count, 256, 0, c.stream>>>(
                                   P, nh, kc, reinterpret_cast<const double2*>(p.d_betar), base)));
  HPSI_LAUNCH(c, HPSI_K_SPLIT,
              (k_split_betar_add<NT><<<4 * c.sm_count, 256, 0, c.stream>>>(P, nr, ka, p.d_betar, base + cal)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "Gamma-form bf16 projector split");
  return HPSI_OK;
}

template <int NT, typename R>
int gamma_apply_tc(Context& c, const Problem& p, const R* x, int nb, bool scaled, int kmax, const float** out,
                   int* nout) {
  const int P = p.nproj, nr = 2 * ((p.npw + 1) / 2);
  const int kc = round_up(nr, TBK), ka = round_up(P, TBK);
  const __nv_bfloat16* bcal = reinterpret_cast<const __nv_bfloat16*>(p.d_betar_bf);
  const __nv_bfloat16* badd = bcal + (size_t)NT * P * kc;
  const int nks = kc / TBK;
  const int tiles = ((nb + TBN - 1) / TBN) * ((P + TBM - 1) / TBM);
  int nsplit = std::max(1, std::min(nks, (2 * c.sm_count + tiles - 1) / tiles));
  int ksplit = std::min((nks + nsplit - 1) / nsplit, kmax);
  nsplit = (nks + ksplit - 1) / ksplit;
  const int naks = ka / TBK;
  const int aksplit = (naks + (naks + kAddKsteps - 1) / kAddKsteps - 1) / ((naks + kAddKsteps - 1) / kAddKsteps);
  const int ansplit = (naks + aksplit - 1) / aksplit;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t xb = al(sizeof(__nv_bfloat16) * (size_t)NT * nb * kc);
  const size_t pb = al(sizeof(float) * (size_t)nsplit * P * nb);
  const size_t wb = al(sizeof(__nv_bfloat16) * (size_t)NT * nb * ka);
  const size_t ab = al(sizeof(float) * (size_t)ansplit * nb * nr);
  const size_t bb = nsplit > 1 ? al(sizeof(double) * (size_t)P * nb) : 0;
  int rc = ensure_buffer(c, &c.ws.mixed, &c.ws.mixedbytes, xb + pb + wb + ab + bb);
  if (rc) return rc;
  unsigned char* w0 = static_cast<unsigned char*>(c.ws.mixed);
  __nv_bfloat16* xs = reinterpret_cast<__nv_bfloat16*>(w0);
  float* part = reinterpret_cast<float*>(w0 + xb);
  __nv_bfloat16* wa = reinterpret_cast<__nv_bfloat16*>(w0 + xb + pb);
  float* apart = reinterpret_cast<float*>(w0 + xb + pb + wb);
  cudaError_t e0 = cudaMemsetAsync(wa, 0, wb, c.stream);   // the K padding of w
  if (e0 != cudaSuccess) return cuda_fail(c, e0, "workspace clear");
  HPSI_LAUNCH(c, HPSI_K_SPLIT,
              (k_split_xr<NT, R><<<dim3(std::min(1024, (kc / 2 + 255) / 256), nb), 256, 0, c.stream>>>(
                  nb, nr, kc, scaled ? 1 : 0, x, xs)));
  rc = launch_gemm<NT>(c, bcal, P, xs, nb, kc, nsplit, ksplit, 0, part, nullptr, 0, HPSI_K_CALBEC);
  if (rc) return rc;
  const int n = P * nb;
  if (nsplit > 1) {
    double* becp = reinterpret_cast<double*>(w0 + xb + pb + wb + ab);
    const size_t nel = (size_t)P * nb;
    HPSI_LAUNCH(c, HPSI_K_DSCALE, (k_sum_partials<<<(int)std::min<size_t>(8 * c.sm_count, (nel + 255) / 256), 256, 0,
                                                    c.stream>>>(nel, nsplit, part, becp)));
    HPSI_LAUNCH(c, HPSI_K_DSCALE,
                (k_dscale_tc_r<NT, double><<<(n + 255) / 256, 256, 0, c.stream>>>(P, nb, 1, ka, becp, p.d_rowptr,
                                                                                  p.d_col, p.d_dvalr, wa)));
  } else {
    HPSI_LAUNCH(c, HPSI_K_DSCALE,
                (k_dscale_tc_r<NT, float><<<(n + 255) / 256, 256, 0, c.stream>>>(P, nb, 1, ka, part, p.d_rowptr,
                                                                                 p.d_col, p.d_dvalr, wa)));
  }
  rc = launch_gemm<NT>(c, wa, nb, badd, nr, ka, ansplit, aksplit, 0, apart, nullptr, 0, HPSI_K_ADDVUS);
  if (rc) return rc;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "Gamma-form tensor-core nonlocal kernels launch");
  *out = apart;
  *nout = ansplit;
  return HPSI_OK;
}

// add_vuspsi on the tensor cores from a float64 w: the complex form (w [nb][P] complex, into hpsi)
// or the real form (w [nb][P] real, float partials [*nout][nb][nr] left in the workspace).  Each
// float32 partial sums one 64-wide K-step: the tensor cores' float32 accumulation is biased (its
// error does not average out in <psi|V_NL psi>, measured 1.3e-6 Ha on the 36785-PW cell at eight
// K-steps per partial), so the quotients this serves get the shortest accumulations, added in
// float64.
template <int NT>
int add_from_w64(Context& c, const Problem& p, const double* w, bool real, int nb, double2* hpsi, const float** out,
                 int* nout) {
  const int P = p.nproj;
  const int kin = real ? P : 2 * P, ka = round_up(kin, TBK);
  const int N = real ? 2 * ((p.npw + 1) / 2) : 2 * p.npw;   // output columns
  const __nv_bfloat16* badd;
  if (real) {
    const int kc = round_up(N, TBK);
    badd = reinterpret_cast<const __nv_bfloat16*>(p.d_betar_bf) + (size_t)NT * P * kc;
  } else {
    badd = reinterpret_cast<const __nv_bfloat16*>(p.d_beta_bf) + (size_t)NT * P * round_up(2 * p.npw, TBK);
  }
  const int naks = ka / TBK;
  const int aksplit = 1, ansplit = naks;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t wb = al(sizeof(__nv_bfloat16) * (size_t)NT * nb * ka);
  const bool partials = real || ansplit > 1;
  const size_t ab = partials ? al(sizeof(float) * (size_t)ansplit * nb * N) : 0;
  int rc = ensure_buffer(c, &c.ws.mixed, &c.ws.mixedbytes, wb + ab);
  if (rc) return rc;
  unsigned char* w0 = static_cast<unsigned char*>(c.ws.mixed);
  __nv_bfloat16* wa = reinterpret_cast<__nv_bfloat16*>(w0);
  float* apart = reinterpret_cast<float*>(w0 + wb);
  HPSI_LAUNCH(c, HPSI_K_SPLIT, (k_split_rows64<NT><<<4 * c.sm_count, 256, 0, c.stream>>>(nb, kin, ka, w, wa)));
  if (partials) {
    rc = launch_gemm<NT>(c, wa, nb, badd, N, ka, ansplit, aksplit, 0, apart, nullptr, 0, HPSI_K_ADDVUS);
    if (rc) return rc;
    if (real) {
      *out = apart;
      *nout = ansplit;
    } else {
      const size_t nel = (size_t)nb * p.npw;
      HPSI_LAUNCH(c, HPSI_K_ADDVUS, (k_add_partials<<<(int)std::min<size_t>(8 * c.sm_count, (nel + 255) / 256), 256,
                                                      0, c.stream>>>(nb, p.npw, ansplit, apart, hpsi)));
    }
  } else {
    rc = launch_gemm<NT>(c, wa, nb, badd, N, ka, 1, naks, 1, nullptr, hpsi, p.npw, HPSI_K_ADDVUS);
    if (rc) return rc;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core add_vuspsi launch");
  return HPSI_OK;
}

}  // namespace

int nonlocal_add_tc(Context& c, const Problem& p, const double2* w, double2* hpsi, int nbnd) {
  if (p.nproj == 0 || nbnd == 0) return HPSI_OK;
  if (!p.d_beta_bf) return fail(c, HPSI_EINVAL, "bf16 projector terms are not prepared");
  const double* wd = reinterpret_cast<const double*>(w);
  return c.nl_terms == 3 ? add_from_w64<3>(c, p, wd, false, nbnd, hpsi, nullptr, nullptr)
                         : add_from_w64<2>(c, p, wd, false, nbnd, hpsi, nullptr, nullptr);
}

int gamma_add_tc(Context& c, const Problem& p, const double* w, int nb, const float** part, int* nsplit) {
  *part = nullptr;
  *nsplit = 0;
  if (p.nproj == 0 || nb == 0) return HPSI_OK;
  if (!p.d_betar_bf) return fail(c, HPSI_EINVAL, "Gamma-form bf16 projector terms are not prepared");
  return c.nl_terms == 3 ? add_from_w64<3>(c, p, w, true, nb, nullptr, part, nsplit)
                         : add_from_w64<2>(c, p, w, true, nb, nullptr, part, nsplit);
}

int gamma_prepare_tc(Context& c, Problem& p) {
  if (p.nproj == 0 || p.d_betar_bf) return HPSI_OK;
  int rc = get_encoder(c);
  if (rc) return rc;
  return c.nl_terms == 3 ? gamma_prepare_t<3>(c, p) : gamma_prepare_t<2>(c, p);
}

int gamma_nonlocal_mixed(Context& c, const Problem& p, const void* x, bool x32, int nb, bool scaled,
                         const float** part, int* nsplit) {
  *part = nullptr;
  *nsplit = 0;
  if (p.nproj == 0 || nb == 0) return HPSI_OK;
  if (!p.d_betar_bf) return fail(c, HPSI_EINVAL, "Gamma-form bf16 projector terms are not prepared");
  const int kmax = c.tc_kmax > 0 ? c.tc_kmax : (p.nl_kmax > 0 ? p.nl_kmax : kCalbecKsteps);
  if (c.nl_terms == 3)
    return x32 ? gamma_apply_tc<3, float>(c, p, static_cast<const float*>(x), nb, scaled, kmax, part, nsplit)
               : gamma_apply_tc<3, double>(c, p, static_cast<const double*>(x), nb, scaled, kmax, part, nsplit);
  return x32 ? gamma_apply_tc<2, float>(c, p, static_cast<const float*>(x), nb, scaled, kmax, part, nsplit)
             : gamma_apply_tc<2, double>(c, p, static_cast<const double*>(x), nb, scaled, kmax, part, nsplit);
}

// Launch the bounded-wait self-test (about 2e6 cycles, ~1 ms).
int wait_selftest(Context& c) {
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON, (k_wait_selftest<<<1, 32, 0, c.stream>>>(c.d_err, 2000000LL)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "self-test launch");
  return HPSI_OK;
}

int mixed_prepare_beta(Context& c, Problem& p) {
  int rc = get_encoder(c);
  if (rc) return rc;
  return c.nl_terms == 3 ? prepare_t<3>(c, p) : prepare_t<2>(c, p);
}

int nonlocal_apply_mixed(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd) {
  if (p.nproj == 0 || nbnd == 0) return HPSI_OK;
  if (c.tc_kmax <= 0 && p.nl_kmax == 0) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c.stream, &cap);
    if (c.autotune && nbnd >= 4 && cap == cudaStreamCaptureStatusNone) {
      const int rc = c.nl_terms == 3 ? tune_ksplit<3>(c, p, psi, nbnd) : tune_ksplit<2>(c, p, psi, nbnd);
      if (rc) return rc;
    }
  }
  const int kmax = c.tc_kmax > 0 ? c.tc_kmax : (p.nl_kmax > 0 ? p.nl_kmax : kCalbecKsteps);
  return c.nl_terms == 3 ? apply_t<3>(c, p, psi, hpsi, nbnd, kmax) : apply_t<2>(c, p, psi, hpsi, nbnd, kmax);
}

void TcInner::release() {
  cudaFree(terms);
  cudaFree(ws);
  *this = TcInner();
}

int tc_inner32(Context& c, TcInner& t, bool cache_a, int rows_cap, const float2* A, int M, const float2* B, int nb,
               int npw, double2* out64, float2* out32, int ldo) {
  constexpr int NT = 3;
  if (M <= 0 || nb <= 0) return HPSI_OK;
  int rc = get_encoder(c);
  if (rc) return rc;
  const int kc = round_up(2 * npw, TBK), nks = kc / TBK;
  const int tiles = ((2 * nb + TBN - 1) / TBN) * ((M + TBM - 1) / TBM);
  // float32 accumulation over at most kInnerKsteps 64-wide K steps, float64 across the splits
  int nsplit = std::max(1, std::min(nks, (2 * c.sm_count + tiles - 1) / tiles));
  int ksplit = std::min((nks + nsplit - 1) / nsplit, c.tc_kmax > 0 ? c.tc_kmax : kInnerKsteps);
  nsplit = (nks + ksplit - 1) / ksplit;
  // workspace: [A split, when not cached][B split][partials], each 256-byte aligned
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t abytes = cache_a ? 0 : al(sizeof(__nv_bfloat16) * NT * (size_t)M * kc);
  const size_t bbytes = al(sizeof(__nv_bfloat16) * NT * (size_t)2 * nb * kc);
  const size_t pbytes = al(sizeof(float) * (size_t)nsplit * M * 2 * nb);
  if (abytes + bbytes + pbytes > t.wsbytes) {
    cudaFree(t.ws);
    t.ws = nullptr;
    t.wsbytes = 0;
    if (cudaMalloc(&t.ws, abytes + bbytes + pbytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, HPSI_ENOMEM, "tensor-core inner-product workspace allocation failed");
    }
    t.wsbytes = abytes + bbytes + pbytes;
  }
  unsigned char* w0 = static_cast<unsigned char*>(t.ws);
  __nv_bfloat16* bsplit = reinterpret_cast<__nv_bfloat16*>(w0 + abytes);
  float* part = reinterpret_cast<float*>(w0 + abytes + bbytes);
  const __nv_bfloat16* asplit;
  size_t pa;
  if (cache_a) {
    // the cached rows stay valid while A, npw and the capacity are unchanged (invalidate() otherwise)
    const int cap = std::max(M, rows_cap);
    if (t.base != A || t.kpad != kc || cap > t.caprows) {
      if (cap > t.caprows) {
        cudaFree(t.terms);
        t.terms = nullptr;
        t.caprows = 0;
        if (cudaMalloc(&t.terms, sizeof(__nv_bfloat16) * NT * (size_t)cap * kc) != cudaSuccess) {
          cudaGetLastError();
          return fail(c, HPSI_ENOMEM, "tensor-core basis split allocation failed");
        }
        t.caprows = cap;
      }
      t.base = A;
      t.kpad = kc;
      t.valid = 0;
    }
    pa = (size_t)t.caprows * kc;
    if (M > t.valid) {
      HPSI_LAUNCH(c, HPSI_K_SPLIT,
                  (k_split_rows32<NT><<<4 * c.sm_count, 256, 0, c.stream>>>(
                      t.valid, M, npw, kc, pa, A, static_cast<__nv_bfloat16*>(t.terms))));
      t.valid = M;
    }
    asplit = static_cast<const __nv_bfloat16*>(t.terms);
  } else {
    pa = (size_t)M * kc;
    __nv_bfloat16* as = reinterpret_cast<__nv_bfloat16*>(w0);
    HPSI_LAUNCH(c, HPSI_K_SPLIT, (k_split_rows32<NT><<<4 * c.sm_count, 256, 0, c.stream>>>(0, M, npw, kc, pa, A, as)));
    asplit = as;
  }
  HPSI_LAUNCH(c, HPSI_K_SPLIT, (k_split_inner_b<NT><<<4 * c.sm_count, 256, 0, c.stream>>>(nb, npw, kc, B, bsplit)));
  rc = launch_gemm<NT>(c, asplit, M, bsplit, 2 * nb, kc, nsplit, ksplit, 0, part, nullptr, 0, HPSI_K_DAVIDSON, pa);
  if (rc) return rc;
  const size_t n = (size_t)M * nb;
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_inner_reduce<<<(int)std::min<size_t>(4 * c.sm_count, (n + 255) / 256), 256, 0, c.stream>>>(
                  M, nb, nsplit, part, out64, out32, ldo)));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "tensor-core inner products launch");
  return HPSI_OK;
}

}  // namespace hpsi
