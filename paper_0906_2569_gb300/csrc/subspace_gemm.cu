// Complex64 products of the mixed-precision Davidson subspace on the bf16 tensor cores.
//
// Every float32 operand x is split into three bf16 terms, x = x0 + x1 + x2 (x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1)), and the products x_i y_j with i + j < 3 (six of
// them, dropping terms below 2^-24 relative) are accumulated in float32 by cuBLAS bf16 GEMMs: the
// result has the accuracy of a float32 product.  A complex matrix stored with interleaved
// (re, im) pairs is read as a real matrix with twice the rows, so no operand is transposed or
// copied into another layout:
//
//   C = A^H B (A: k x m, B: k x n):  P = Ar^T [Br | B~r] (m x 2n), Re C = P[:, b], Im C = P[:, n+b],
//       with Ar, Br the real (2k x .) views and B~ = (Im B, -Re B) interleaved;
//   C = A B (A: M x k, B: k x n):    P = Ar [Re B | Im B] (2M x 2n),
//       Re C[g][b] = P[2g][b] - P[2g+1][n+b],  Im C[g][b] = P[2g][n+b] + P[2g+1][b].
//
// The large operand (the basis phi or H phi) keeps its split in a cache that is extended column
// by column as the basis grows; the small operand is split per call.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "hpsi_internal.h"

namespace hpsi {

namespace {

__device__ __forceinline__ void split3(float x, __nv_bfloat16* t0, __nv_bfloat16* t1, __nv_bfloat16* t2) {
  const __nv_bfloat16 a = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(a);
  const __nv_bfloat16 b = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(b);
  *t0 = a;
  *t1 = b;
  *t2 = __float2bfloat16_rn(r2);
}

// Split n floats (a contiguous range) into three bf16 arrays at the same offsets.
__global__ void k_split_range(size_t n, const float* __restrict__ x, __nv_bfloat16* __restrict__ t0,
                              __nv_bfloat16* __restrict__ t1, __nv_bfloat16* __restrict__ t2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    split3(x[i], t0 + i, t1 + i, t2 + i);
}

// B (k x n complex64, ldb) -> [Br | B~r] (2k x 2n real, ld 2k), split.
__global__ void k_prep_ah(int k, int n, const float2* __restrict__ B, int ldb, __nv_bfloat16* __restrict__ t0,
                          __nv_bfloat16* __restrict__ t1, __nv_bfloat16* __restrict__ t2) {
  const size_t total = (size_t)k * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(i % k), b = (int)(i / k);
    const float2 v = B[(size_t)b * ldb + g];
    const size_t o0 = (size_t)b * 2 * k + 2 * g, o1 = (size_t)(n + b) * 2 * k + 2 * g;
    split3(v.x, t0 + o0, t1 + o0, t2 + o0);
    split3(v.y, t0 + o0 + 1, t1 + o0 + 1, t2 + o0 + 1);
    split3(v.y, t0 + o1, t1 + o1, t2 + o1);
    split3(-v.x, t0 + o1 + 1, t1 + o1 + 1, t2 + o1 + 1);
  }
}

// B (k x n complex64, ldb) -> [Re B | Im B] (k x 2n real, ld k), split.
__global__ void k_prep_ab(int k, int n, const float2* __restrict__ B, int ldb, __nv_bfloat16* __restrict__ t0,
                          __nv_bfloat16* __restrict__ t1, __nv_bfloat16* __restrict__ t2) {
  const size_t total = (size_t)k * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i % k), b = (int)(i / k);
    const float2 v = B[(size_t)b * ldb + r];
    const size_t o0 = (size_t)b * k + r, o1 = (size_t)(n + b) * k + r;
    split3(v.x, t0 + o0, t1 + o0, t2 + o0);
    split3(v.y, t0 + o1, t1 + o1, t2 + o1);
  }
}

// C (m x n) = alpha (P[:, b] + i P[:, n+b]) + beta C, P (m x 2n, ld m) float32.
template <typename T>
__global__ void k_fix_ah(int m, int n, const float* __restrict__ P, float alpha, float beta, T* __restrict__ C,
                         int ldc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * n) return;
  const int r = i % m, b = i / m;
  const float re = P[(size_t)b * m + r], im = P[(size_t)(n + b) * m + r];
  T& c = C[(size_t)b * ldc + r];
  if (beta == 0.f) {
    c.x = alpha * re;
    c.y = alpha * im;
  } else {
    c.x = alpha * re + beta * c.x;
    c.y = alpha * im + beta * c.y;
  }
}

// C (M x n complex64) = alpha (A B) + beta C from P (2M x 2n, ld 2M) float32.
__global__ void k_fix_ab(int M, int n, const float* __restrict__ P, float alpha, float beta, float2* __restrict__ C,
                         int ldc) {
  const size_t total = (size_t)M * n;
  const size_t ld = 2 * (size_t)M;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int g = (int)(i % M), b = (int)(i / M);
    const float p00 = P[(size_t)b * ld + 2 * g], p10 = P[(size_t)b * ld + 2 * g + 1];
    const float p01 = P[(size_t)(n + b) * ld + 2 * g], p11 = P[(size_t)(n + b) * ld + 2 * g + 1];
    float2& c = C[(size_t)b * ldc + g];
    const float re = p00 - p11, im = p01 + p10;
    if (beta == 0.f) {
      c = make_float2(alpha * re, alpha * im);
    } else {
      c = make_float2(alpha * re + beta * c.x, alpha * im + beta * c.y);
    }
  }
}

int grid_for(size_t n) { return (int)std::min<size_t>(8192, (n + 255) / 256); }

// P = sum_{i + j < 3} op(A_i) B_j, float32 (six cuBLAS bf16 GEMMs, smallest terms first)
int six_products(Context& c, cublasHandle_t h, cublasOperation_t ta, int m, int n, int k,
                 __nv_bfloat16* const* A, int lda, __nv_bfloat16* const* B, int ldb, float* P, int ldp) {
  static const int order[6][2] = {{2, 0}, {1, 1}, {0, 2}, {1, 0}, {0, 1}, {0, 0}};
  const float one = 1.f, zero = 0.f;
  for (int t = 0; t < 6; ++t) {
    const cublasStatus_t st =
        cublasGemmEx(h, ta, CUBLAS_OP_N, m, n, k, &one, A[order[t][0]], CUDA_R_16BF, lda, B[order[t][1]], CUDA_R_16BF,
                     ldb, t == 0 ? &zero : &one, P, CUDA_R_32F, ldp, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    if (st != CUBLAS_STATUS_SUCCESS) return fail(c, HPSI_ECUDA, "bf16 subspace GEMM failed");
  }
  return HPSI_OK;
}

}  // namespace

int SplitBasis::ensure(Context& c, const float2* src, int ld, int cols) {
  if (src != base || ld != lds) {
    base = src;
    lds = ld;
    valid = 0;
  }
  const size_t need = (size_t)2 * ld * cols;
  if (need > cap) {
    for (auto& t : terms) cudaFree(t);
    terms[0] = terms[1] = terms[2] = nullptr;
    for (auto& t : terms)
      if (cudaMalloc((void**)&t, sizeof(__nv_bfloat16) * need) != cudaSuccess)
        return fail(c, HPSI_ENOMEM, "bf16 basis split allocation failed");
    cap = need;
    valid = 0;
  }
  if (cols > valid) {
    const size_t off = (size_t)2 * ld * valid, cnt = (size_t)2 * ld * (cols - valid);
    k_split_range<<<grid_for(cnt), 256, 0, c.stream>>>(cnt, reinterpret_cast<const float*>(src) + off,
                                                       terms[0] + off, terms[1] + off, terms[2] + off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "basis split");
    valid = cols;
  }
  return HPSI_OK;
}

void SplitBasis::release() {
  for (auto& t : terms) cudaFree(t);
  terms[0] = terms[1] = terms[2] = nullptr;
  cap = 0;
  valid = 0;
  base = nullptr;
}

int SubspaceGemm::grow(Context& c, size_t bterms, size_t pfloats) {
  if (bterms > bcap) {
    for (auto& t : bt) cudaFree(t);
    bt[0] = bt[1] = bt[2] = nullptr;
    for (auto& t : bt)
      if (cudaMalloc((void**)&t, sizeof(__nv_bfloat16) * bterms) != cudaSuccess)
        return fail(c, HPSI_ENOMEM, "bf16 operand split allocation failed");
    bcap = bterms;
  }
  if (pfloats > pcap) {
    cudaFree(P);
    P = nullptr;
    if (cudaMalloc((void**)&P, sizeof(float) * pfloats) != cudaSuccess)
      return fail(c, HPSI_ENOMEM, "subspace GEMM workspace allocation failed");
    pcap = pfloats;
  }
  return HPSI_OK;
}

void SubspaceGemm::release() {
  for (auto& t : bt) cudaFree(t);
  cudaFree(P);
  bt[0] = bt[1] = bt[2] = nullptr;
  P = nullptr;
  bcap = pcap = 0;
}

int SubspaceGemm::ah_b(Context& c, cublasHandle_t h, int m, int n, int k, SplitBasis& A, const float2* Asrc, int lda,
                       const float2* B, int ldb, float alpha, float beta, float2* C32, double2* C64, int ldc) {
  if (m <= 0 || n <= 0) return HPSI_OK;
  int rc = A.ensure(c, Asrc, lda, m);
  if (rc) return rc;
  rc = grow(c, (size_t)2 * k * 2 * n, (size_t)m * 2 * n);
  if (rc) return rc;
  k_prep_ah<<<grid_for((size_t)k * n), 256, 0, c.stream>>>(k, n, B, ldb, bt[0], bt[1], bt[2]);
  rc = six_products(c, h, CUBLAS_OP_T, m, 2 * n, 2 * k, A.terms, 2 * lda, bt, 2 * k, P, m);
  if (rc) return rc;
  if (C64)
    k_fix_ah<double2><<<(m * n + 255) / 256, 256, 0, c.stream>>>(m, n, P, alpha, beta, C64, ldc);
  else
    k_fix_ah<float2><<<(m * n + 255) / 256, 256, 0, c.stream>>>(m, n, P, alpha, beta, C32, ldc);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HPSI_OK : cuda_fail(c, e, "subspace GEMM epilogue");
}

int SubspaceGemm::a_b(Context& c, cublasHandle_t h, int M, int n, int k, SplitBasis& A, const float2* Asrc, int lda,
                      const float2* B, int ldb, float alpha, float beta, float2* C, int ldc) {
  if (n <= 0 || M <= 0) return HPSI_OK;
  int rc = A.ensure(c, Asrc, lda, k);
  if (rc) return rc;
  rc = grow(c, (size_t)k * 2 * n, (size_t)2 * M * 2 * n);
  if (rc) return rc;
  k_prep_ab<<<grid_for((size_t)k * n), 256, 0, c.stream>>>(k, n, B, ldb, bt[0], bt[1], bt[2]);
  rc = six_products(c, h, CUBLAS_OP_N, 2 * M, 2 * n, k, A.terms, 2 * lda, bt, k, P, 2 * M);
  if (rc) return rc;
  k_fix_ab<<<grid_for((size_t)M * n), 256, 0, c.stream>>>(M, n, P, alpha, beta, C, ldc);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HPSI_OK : cuda_fail(c, e, "subspace GEMM epilogue");
}

}  // namespace hpsi
