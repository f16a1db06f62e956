// hpsi_apply_noalloc: H|psi> without any device allocation at call time.
//
// Some callers cannot let a library call cudaMalloc: their device memory is reserved up front
// by another allocator (a framework's caching pool, a fixed per-process budget), or they cannot
// accept the device-wide synchronisation that cudaMalloc / cudaFree imply in the middle of an
// asynchronous stream pipeline.  This entry point computes the same H|psi> as hpsi_apply, but
// every intermediate (the plane and stick buffers of the FFTs, the partial sums of <beta|psi>
// and D<beta|psi>) lives in one fixed array compiled into the library.  Bands are processed in
// chunks that fit the array.  The local term runs on the register-codelet kernels where the box
// has them (with the plan chosen at setup or by an earlier hpsi_apply), else on the generic ones;
// the nonlocal term runs on the float64 kernels at either precision (they need no buffers beyond
// the array).
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "hpsi_internal.h"

namespace {

// 64 MiB, 256-byte aligned.  Every GPU that loads libhpsi.so holds it until the process exits.
constexpr size_t kNoAllocBytes = size_t(64) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the array on the context's device, looked up once per device with that
// device current (the caller's current device is restored).  The host-side name g_noalloc_scratch
// is only a stand-in: kernels must be given this address instead.
int scratch_address(hpsi::Context& c, void** out) {
  const int dev = c.device;
  if (dev < 0 || dev >= kMaxDevices) return hpsi::fail(c, HPSI_ENODEV, "hpsi_apply_noalloc: device index too large");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return hpsi::cuda_fail(c, e, "hpsi_apply_noalloc: cudaGetDevice");
    if (prev != dev && (e = cudaSetDevice(dev)) != cudaSuccess)
      return hpsi::cuda_fail(c, e, "hpsi_apply_noalloc: cudaSetDevice");
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess || !p) return hpsi::cuda_fail(c, e, "hpsi_apply_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return HPSI_OK;
}

bool on_device(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int hpsi_apply_noalloc(hpsi_ctx* ctx, int ik, const void* psi_in, void* hpsi_out, int nbnd) {
  if (!ctx) return HPSI_EINVAL;
  hpsi::Context& c = ctx->c;
  if (ik < 0 || ik >= (int)c.probs.size()) return hpsi::fail(c, HPSI_EINVAL, "hpsi_apply_noalloc: problem index out of range");
  if (nbnd < 0) return hpsi::fail(c, HPSI_EINVAL, "hpsi_apply_noalloc: nbnd < 0");
  if (nbnd == 0) return HPSI_OK;
  if (!psi_in || !hpsi_out) return hpsi::fail(c, HPSI_EINVAL, "hpsi_apply_noalloc: null pointer");
  const hpsi::Problem& p = c.probs[ik];
  const size_t bytes = sizeof(double2) * (size_t)nbnd * p.npw;
  const char* a0 = static_cast<const char*>(psi_in);
  const char* b0 = static_cast<const char*>(hpsi_out);
  if (a0 < b0 + bytes && b0 < a0 + bytes) return hpsi::fail(c, HPSI_EINVAL, "hpsi_apply_noalloc: psi_in and hpsi_out overlap");
  if (!on_device(psi_in) || !on_device(hpsi_out))
    return hpsi::fail(c, HPSI_EINVAL, "hpsi_apply_noalloc: psi_in and hpsi_out must be device memory");
  void* base = nullptr;
  int rc = scratch_address(c, &base);
  if (rc) return rc;
  // Largest band chunk whose X and Y and the nonlocal partials fit the array.  X and Y of a chunk
  // scale with its bands, so a shorter last chunk fits in the same places; its nonlocal K-split
  // is planned against the room left after the full chunk's X and Y, and one split of the partials
  // grows with the bands too, so whatever fits the full chunk fits the last one.
  // The register-codelet kernels (cubic boxes with a two-factor edge) need two stick-row buffers per
  // band; the generic kernels an m1-plane buffer and a stick-row buffer.
  const int prec = hpsi::cur_prec(c);
  const bool fast = (p.fflags[prec] & 4) && !c.force_generic;
  const size_t cs = prec == HPSI_FP64 ? sizeof(double2) : sizeof(float2);
  auto xbytes = [&](int nb) {
    return align256(cs * (size_t)nb * p.n[2] * (fast ? (size_t)p.nst : (size_t)p.npl * p.n[1]));
  };
  auto ybytes = [&](int nb) { return align256(cs * (size_t)nb * p.n[2] * p.nst); };
  const size_t per_band = xbytes(1) + ybytes(1);
  int chunk = 0;
  for (int nb = std::min(nbnd, 4096); nb >= 1; nb = nb > 64 ? nb - 32 : nb - 1) {
    const size_t xy = xbytes(nb) + ybytes(nb);
    if (xy > kNoAllocBytes) continue;
    int ns = 0, kc = 0;
    size_t nl = 0;
    hpsi::nonlocal_fp64_plan(c, p, nb, &ns, &kc, &nl);
    if (p.nproj == 0 || xy + align256(nl) <= kNoAllocBytes) {
      chunk = nb;
      break;
    }
  }
  if (chunk == 0)
    return hpsi::fail(c, HPSI_EINVAL,
                      "hpsi_apply_noalloc: one band needs " + std::to_string(per_band) +
                          " bytes of intermediates, more than the fixed 64 MiB array; use hpsi_apply");
  unsigned char* s = static_cast<unsigned char*>(base);
  void* X = s;
  void* Y = s + xbytes(chunk);
  void* NL = static_cast<unsigned char*>(Y) + ybytes(chunk);
  const size_t nl_room = kNoAllocBytes - xbytes(chunk) - ybytes(chunk);
  const double2* psi = static_cast<const double2*>(psi_in);
  double2* hpsi = static_cast<double2*>(hpsi_out);
  for (int b = 0; b < nbnd; b += chunk) {
    const int nb = std::min(chunk, nbnd - b);
    if (xbytes(nb) > xbytes(chunk) || ybytes(nb) > ybytes(chunk))
      return hpsi::fail(c, HPSI_EINVAL, "hpsi_apply_noalloc: internal chunk sizing error");
    rc = fast ? hpsi::local_fast_apply(c, p, psi + (size_t)b * p.npw, hpsi + (size_t)b * p.npw, nb, X, Y, nb)
              : hpsi::local_apply_into(c, p, psi + (size_t)b * p.npw, hpsi + (size_t)b * p.npw, nb, X, Y, nb);
    if (rc) return rc;
    rc = hpsi::nonlocal_fp64_into(c, p, psi + (size_t)b * p.npw, hpsi + (size_t)b * p.npw, nb, NL, nl_room);
    if (rc) return rc;
    c.band_apps += nb;
  }
  return HPSI_OK;
}
