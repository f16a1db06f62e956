// Dependent-chain latency of float64 (and, for comparison, float32 and integer) operations on one
// GPU, and float64 FMA throughput of one SM as the number of warps and independent chains grows.
// Every kernel runs a fixed, bounded number of iterations on one CTA and times itself with clock64.
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("err %s line %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

enum Op { DFMA, DADD, DMUL, DDIV, DSQRT, DSHFL, FFMA, IADD };

template <int OP>
__global__ void chain(double* out, long long* cyc, int iters, double a, double b) {
  double x = 1.0 + threadIdx.x * 1e-9;
  float xf = (float)x;
  int xi = threadIdx.x;
  __syncwarp();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (OP == DFMA) x = fma(x, a, b);
      if (OP == DADD) x = x + b;
      if (OP == DMUL) x = x * a;
      if (OP == DDIV) x = b / x + a;
      if (OP == DSQRT) x = sqrt(x) + b;
      if (OP == DSHFL) x = __shfl_xor_sync(0xffffffffu, x, 1) + b;
      if (OP == FFMA) xf = fmaf(xf, (float)a, (float)b);
      if (OP == IADD) xi = xi * 3 + 1;
    }
  }
  const long long t1 = clock64();
  out[threadIdx.x] = x + xf + xi;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

// NC independent DFMA chains per thread
template <int NC>
__global__ void dfma_tput(double* out, long long* cyc, int iters, double a, double b) {
  double x[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) x[c] = 1.0 + c + threadIdx.x * 1e-9;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
#pragma unroll
      for (int c = 0; c < NC; ++c) x[c] = fma(x[c], a, b);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < NC; ++c) s += x[c];
  out[threadIdx.x] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

template <int OP>
int run_chain(const char* name, double* out, long long* cyc, int threads) {
  const int iters = 256;
  long long h = 0;
  chain<OP><<<1, threads>>>(out, cyc, iters, 0.999999, 1e-7);
  CK(cudaDeviceSynchronize());
  chain<OP><<<1, threads>>>(out, cyc, iters, 0.999999, 1e-7);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost));
  printf("  %-6s threads %4d : %7.1f cycles per dependent op\n", name, threads, (double)h / (iters * 8));
  return 0;
}

template <int NC>
int run_tput(double* out, long long* cyc, int warps) {
  const int iters = 128;
  long long h = 0;
  dfma_tput<NC><<<1, 32 * warps>>>(out, cyc, iters, 0.999999, 1e-7);
  CK(cudaDeviceSynchronize());
  dfma_tput<NC><<<1, 32 * warps>>>(out, cyc, iters, 0.999999, 1e-7);
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost));
  const double ops = (double)iters * 8 * NC * 32 * warps;
  printf("  DFMA throughput, %2d warps x %d chains/thread : %6.3f lane-FMA per cycle per SM\n", warps, NC, ops / h);
  return 0;
}

int main() {
  double* out;
  long long* cyc;
  CK(cudaMalloc(&out, sizeof(double) * 1024));
  CK(cudaMalloc(&cyc, sizeof(long long) * 8));
  printf("dependent-chain latency (one CTA):\n");
  for (int t : {1, 32}) {
    if (run_chain<DFMA>("DFMA", out, cyc, t) || run_chain<DADD>("DADD", out, cyc, t) ||
        run_chain<DMUL>("DMUL", out, cyc, t) || run_chain<DDIV>("DDIV", out, cyc, t) ||
        run_chain<DSQRT>("DSQRT", out, cyc, t) || (t == 32 && run_chain<DSHFL>("SHFL+D", out, cyc, t)) ||
        run_chain<FFMA>("FFMA", out, cyc, t) || run_chain<IADD>("IMAD", out, cyc, t))
      return 1;
  }
  printf("float64 FMA throughput of one SM:\n");
  for (int w : {1, 4, 8, 16, 32}) {
    if (run_tput<1>(out, cyc, w) || run_tput<4>(out, cyc, w) || run_tput<8>(out, cyc, w)) return 1;
  }
  return 0;
}
