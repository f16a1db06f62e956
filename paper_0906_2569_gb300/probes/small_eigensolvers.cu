// Timing of cuSOLVER small Hermitian eigensolvers (zheevd, zheevdx for the lowest quarter, zheevj)
// at the reduced-matrix sizes of the Davidson solver (160 ... 2048).
#include <cusolverDn.h>
#include <cuda_runtime.h>
#include <cstdio>
#include <vector>
#include <random>
#define CK(x) do{int e=(int)(x); if(e){printf("err %d line %d\n",e,__LINE__); return 1;}}while(0)
int main() {
  cusolverDnHandle_t h; CK(cusolverDnCreate(&h));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  for (int n : {160, 320, 640, 1280, 2048}) {
    std::vector<cuDoubleComplex> A((size_t)n * n);
    std::mt19937_64 g(n); std::normal_distribution<double> d(0, 1);
    for (int j = 0; j < n; ++j) for (int i = 0; i <= j; ++i) {
      cuDoubleComplex v = make_cuDoubleComplex(d(g), i == j ? 0 : d(g));
      A[(size_t)j * n + i] = v; A[(size_t)i * n + j] = make_cuDoubleComplex(v.x, -v.y);
    }
    cuDoubleComplex *dA, *dW0, *work; double* W; int* info;
    CK(cudaMalloc(&dA, A.size() * 16)); CK(cudaMalloc(&dW0, A.size() * 16)); CK(cudaMalloc(&W, n * 8)); CK(cudaMalloc(&info, 4));
    CK(cudaMemcpy(dW0, A.data(), A.size() * 16, cudaMemcpyHostToDevice));
    int lw = 0;
    CK(cusolverDnZheevd_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, dA, n, W, &lw));
    int lw2 = 0, meig = 0;
    CK(cusolverDnZheevdx_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_UPPER, n, dA, n, 0, 0, 1, n / 4, &meig, W, &lw2));
    syevjInfo_t params; CK(cusolverDnCreateSyevjInfo(&params));
    int lw3 = 0;
    CK(cusolverDnZheevj_bufferSize(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, dA, n, W, &lw3, params));
    int lwm = std::max(lw, std::max(lw2, lw3));
    CK(cudaMalloc(&work, (size_t)lwm * 16));
    for (int mode = 0; mode < 3; ++mode) {
      float best = 1e9;
      for (int rep = 0; rep < 3; ++rep) {
        CK(cudaMemcpy(dA, dW0, A.size() * 16, cudaMemcpyDeviceToDevice));
        cudaEventRecord(e0);
        if (mode == 0) CK(cusolverDnZheevd(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, dA, n, W, work, lw, info));
        if (mode == 1) CK(cusolverDnZheevdx(h, CUSOLVER_EIG_MODE_VECTOR, CUSOLVER_EIG_RANGE_I, CUBLAS_FILL_MODE_UPPER, n, dA, n, 0, 0, 1, n / 4, &meig, W, work, lw2, info));
        if (mode == 2) CK(cusolverDnZheevj(h, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, n, dA, n, W, work, lw3, info, params));
        cudaEventRecord(e1); cudaEventSynchronize(e1);
        float ms; cudaEventElapsedTime(&ms, e0, e1); if (ms < best) best = ms;
      }
      printf("n=%5d %s: %.3f ms\n", n, mode == 0 ? "zheevd " : mode == 1 ? "zheevdx(n/4)" : "zheevj ", best);
    }
    cudaFree(dA); cudaFree(dW0); cudaFree(W); cudaFree(info); cudaFree(work); cusolverDnDestroySyevjInfo(params);
  }
  return 0;
}
