// Grid-barrier cost on one GPU: cooperative launch, G CTAs x 256 threads, every wait bounded (about
// 1 s, then an error flag).  Mode 0: one counter, red.release add + ld.acquire polling (the barrier of
// the tridiagonal reduction); mode 1: one release flag per CTA, polled by G threads of every CTA;
// modes 2 and 3: the same with an all-gather of n = 400 complex values through L2 per barrier, as the
// reduction does with y each column.
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o grid_barrier grid_barrier.cu
#include <cstdio>
#include <cuda_runtime.h>
#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("err %s line %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)
constexpr long long kLimit = 2000000000LL;

__device__ bool wait_counter(unsigned* count, unsigned target, int* err) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    int good = 1; const long long t0 = clock64(); unsigned spins = 0;
    for (;;) {
      unsigned v; asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if ((int)(v - target) >= 0) break;
      if ((++spins & 255u) == 0u && (*(volatile int*)err != 0 || clock64() - t0 > kLimit)) { atomicCAS(err, 0, 3); good = 0; break; }
    }
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}
// flags[g] = epoch (release store); warps 0..(G+31)/32-1 poll all flags
__device__ bool wait_flags(unsigned* flags, int G, unsigned target, int* err) {
  __shared__ int ok;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  const int i = threadIdx.x;
  if (i < G) {
    const long long t0 = clock64(); unsigned spins = 0;
    for (;;) {
      unsigned v; asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flags + i) : "memory");
      if ((int)(v - target) >= 0) break;
      if ((++spins & 255u) == 0u && (*(volatile int*)err != 0 || clock64() - t0 > kLimit)) { atomicCAS(err, 0, 3); ok = 0; break; }
    }
  }
  __syncthreads();
  return ok != 0;
}

// mode 0: counter barrier; 1: flag barrier; 2: counter + all-gather of n double2; 3: flags + all-gather
__global__ void probe(int mode, int iters, int n, unsigned* bar, unsigned* flags, double2* buf, double* out, long long* cyc, int* err) {
  const int G = gridDim.x, g = blockIdx.x;
  double acc = 0.0;
  __syncthreads();
  const long long t0 = clock64();
  for (int j = 0; j < iters; ++j) {
    if (mode >= 2) {   // write own rows' values of this epoch
      for (int r = g + threadIdx.x * G; r < n; r += G * blockDim.x)
        buf[(j & 1) * n + r] = make_double2(r + j, g);
    }
    __syncthreads();
    if (mode == 0 || mode == 2) {
      if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
      if (!wait_counter(bar, (unsigned)(G * (j + 1)), err)) break;
    } else {
      if (threadIdx.x == 0) asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flags + g), "r"(j + 1) : "memory");
      if (!wait_flags(flags, G, (unsigned)(j + 1), err)) break;
    }
    if (mode >= 2) {
      for (int c = threadIdx.x; c < n; c += blockDim.x) acc += __ldcg(&buf[(j & 1) * n + c]).x;
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cyc[g] = t1 - t0;
  out[g * blockDim.x + threadIdx.x] = acc;
}

int main() {
  int dev = 0; cudaDeviceProp prop; CK(cudaGetDeviceProperties(&prop, dev));
  const int SM = prop.multiProcessorCount;
  unsigned *bar, *flags; double2* buf; double* out; long long* cyc; int* err;
  CK(cudaMalloc(&bar, 64 * sizeof(unsigned))); CK(cudaMalloc(&flags, 256 * sizeof(unsigned)));
  CK(cudaMalloc(&buf, 2 * 1024 * sizeof(double2))); CK(cudaMalloc(&out, 256 * 256 * sizeof(double)));
  CK(cudaMalloc(&cyc, 256 * sizeof(long long))); CK(cudaMalloc(&err, sizeof(int)));
  int nb = 0; CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, probe, 256, 0));
  printf("SMs %d, resident CTAs per SM %d\n", SM, nb);
  const int iters = 2000, n = 400;
  for (int G : {SM, SM / 2, SM / 4, 16}) {
    if (G > SM * nb || G > 256) continue;
    for (int mode = 0; mode < 4; ++mode) {
      for (int rep = 0; rep < 2; ++rep) {
        CK(cudaMemset(bar, 0, 64 * sizeof(unsigned))); CK(cudaMemset(flags, 0, 256 * sizeof(unsigned))); CK(cudaMemset(err, 0, sizeof(int)));
        int m = mode, it = iters, nn = n;
        void* args[] = {&m, &it, &nn, &bar, &flags, &buf, &out, &cyc, &err};
        cudaEvent_t e0, e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0));
        CK(cudaLaunchCooperativeKernel((const void*)probe, dim3(G), dim3(256), args, 0, 0));
        CK(cudaEventRecord(e1)); CK(cudaEventSynchronize(e1));
        float ms = 0; CK(cudaEventElapsedTime(&ms, e0, e1));
        int herr = 0; CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
        long long hc = 0; CK(cudaMemcpy(&hc, cyc, sizeof(long long), cudaMemcpyDeviceToHost));
        if (rep == 1)
          printf("G %3d mode %d (%s%s): %6.2f us per barrier (events), %7.0f cycles (CTA 0), err %d\n", G, mode,
                 (mode & 1) ? "flags" : "counter", mode >= 2 ? " + all-gather n=400" : "", ms * 1e3 / iters, (double)hc / iters, herr);
        if (herr) return 2;
      }
    }
  }
  return 0;
}
