// Full-box 3-D transforms of grid functions, and the maps between the G-sphere and the box.  Used
// where a whole grid function is needed (the density, the Hartree potential, codensities of the
// exchange operator) rather than the sphere-pruned passes of H|psi>.  Boxes are [n3][n2][n1]
// complex128 with x fastest, several in a row (box b at b * n1 n2 n3); each line is transformed by
// one warp with the shared-memory line transform of the local kernels (warp_fft.cuh).
#pragma once

#include <cuda_runtime.h>

#include "hpsi_internal.h"
#include "warp_fft.cuh"

namespace hpsi {

// One line per warp along an axis of box blockIdx.y.  DIR = +1: sum_m a(m) e^{+2 pi i m j / n};
// DIR = -1: the same sum with e^{-i}.  Shared memory: 8 lines of plan.n complex128.
template <int DIR>
__global__ void __launch_bounds__(256) k_box_fft(double2* __restrict__ boxes, int n1, int n2, int n3, int axis,
                                                 FftPlan plan, int nlines) {
  extern __shared__ __align__(16) unsigned char box_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int line = blockIdx.x * kWarpsPerCta + warp;
  if (line >= nlines) return;   // uniform per warp; the line transform synchronises only its warp
  double2* box = boxes + (size_t)blockIdx.y * n1 * n2 * n3;
  const int n = plan.n;
  double2* L = reinterpret_cast<double2*>(box_smem) + (size_t)warp * n;
  size_t base, stride;
  if (axis == 0) {
    base = (size_t)line * n1;
    stride = 1;
  } else if (axis == 1) {
    const int j3 = line / n1, j1 = line - j3 * n1;
    base = (size_t)j3 * n2 * n1 + j1;
    stride = n1;
  } else {
    base = line;
    stride = (size_t)n1 * n2;
  }
  for (int i = lane; i < n; i += 32) L[i] = box[base + i * stride];
  __syncwarp();
  warp_fft<DIR>(L, plan, lane);
  for (int i = lane; i < n; i += 32) box[base + i * stride] = L[i];
}

// The three axes of nbox boxes of problem p, in the direction dir (+1 or -1).
inline int box_fft(Context& c, const Problem& p, double2* boxes, int nbox, int dir, int kclass) {
  const int n1 = p.n[0], n2 = p.n[1], n3 = p.n[2];
  const int nlines[3] = {n2 * n3, n1 * n3, n1 * n2};
  for (int a = 0; a < 3; ++a) {
    const size_t smem = sizeof(double2) * (size_t)kWarpsPerCta * p.n[a];
    const dim3 grid((nlines[a] + kWarpsPerCta - 1) / kWarpsPerCta, nbox);
    if (dir > 0)
      HPSI_LAUNCH(c, kclass, (k_box_fft<+1><<<grid, 256, smem, c.stream>>>(boxes, n1, n2, n3, a, p.plan[a], nlines[a])));
    else
      HPSI_LAUNCH(c, kclass, (k_box_fft<-1><<<grid, 256, smem, c.stream>>>(boxes, n1, n2, n3, a, p.plan[a], nlines[a])));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "box transform");
  return HPSI_OK;
}

}  // namespace hpsi
