// Throughput microbenchmark for the roofline denominators: FP64 FMA, FP32 FMA and FP64 MMA
// (mma.sync m8n8k4) rates of one GPU, with independent accumulation chains; bounded loops.
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do{cudaError_t e=(x); if(e!=cudaSuccess){printf("err %s line %d\n",cudaGetErrorString(e),__LINE__); return 1;}}while(0)

template<typename T>
__global__ void fma_loop(T* out, int iters, T a, T b) {
  T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0+4, x5=x0+5, x6=x0+6, x7=x0+7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

__global__ void dmma_loop(double* out, int iters) {
  double a = threadIdx.x * 1e-3, b = 0.5;
  double c0 = 0, c1 = 0, c2 = 0, c3 = 0, d0=0, d1=0, e0=0,e1=0;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c0), "+d"(c1) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(c2), "+d"(c3) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(d0), "+d"(d1) : "d"(a), "d"(b));
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
                   : "+d"(e0), "+d"(e1) : "d"(a), "d"(b));
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = c0 + c1 + c2 + c3 + d0 + d1 + e0 + e1;
}

int main() {
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, 0));
  printf("name %s SMs %d cc %d.%d l2 %d smemPerBlockOptin %zu smemPerSM %zu regsPerSM %d clock(kHz) %d\n",
         p.name, p.multiProcessorCount, p.major, p.minor, p.l2CacheSize, p.sharedMemPerBlockOptin,
         p.sharedMemPerMultiprocessor, p.regsPerMultiprocessor, 0);
  int sms = p.multiProcessorCount;
  double* dout; float* fout; CK(cudaMalloc(&dout, sizeof(double) * sms * 8 * 1024)); CK(cudaMalloc(&fout, sizeof(float) * sms * 8 * 1024));
  cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
  int blocks = sms * 4, threads = 512;
  for (int rep = 0; rep < 2; ++rep) {
    int iters = 2000;
    fma_loop<double><<<blocks, threads>>>(dout, 10, 1.0000001, 1e-7); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); fma_loop<double><<<blocks, threads>>>(dout, iters, 1.0000001, 1e-7); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    float ms; cudaEventElapsedTime(&ms, e0, e1);
    double flops = 2.0 * 16 * 8 * (double)iters * blocks * threads;
    printf("DFMA: %.3f TFLOP/s (%.2f ms)\n", flops / ms / 1e9, ms);
    iters = 20000;
    fma_loop<float><<<blocks, threads>>>(fout, 10, 1.0000001f, 1e-7f); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); fma_loop<float><<<blocks, threads>>>(fout, iters, 1.0000001f, 1e-7f); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    flops = 2.0 * 16 * 8 * (double)iters * blocks * threads;
    printf("FFMA: %.3f TFLOP/s (%.2f ms)\n", flops / ms / 1e9, ms);
    iters = 500;
    dmma_loop<<<blocks, 256>>>(dout, 10); CK(cudaDeviceSynchronize());
    cudaEventRecord(e0); dmma_loop<<<blocks, 256>>>(dout, iters); cudaEventRecord(e1); CK(cudaEventSynchronize(e1));
    cudaEventElapsedTime(&ms, e0, e1);
    // per warp per mma: 8x8x4 MACs = 512 flops
    flops = 512.0 * 32 * (double)iters * blocks * (256 / 32);
    printf("DMMA m8n8k4: %.3f TFLOP/s (%.2f ms)\n", flops / ms / 1e9, ms);
  }
  CK(cudaGetLastError());
  return 0;
}
