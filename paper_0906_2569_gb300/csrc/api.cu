// extern "C" entry points of libhpsi (declared and documented in include/hpsi.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>

#include "hpsi_internal.h"

namespace hpsi {

static thread_local std::string g_setup_err;

int fail(Context& c, int code, const std::string& msg) {
  c.err = msg;
  return code;
}

int cuda_fail(Context& c, cudaError_t e, const char* what) {
  c.err = std::string(what) + ": " + cudaGetErrorString(e);
  return HPSI_ECUDA;
}

static cudaEvent_t pooled_event(Context& c) {
  if (!c.evpool.empty()) {
    cudaEvent_t e = c.evpool.back();
    c.evpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int launch_begin(Context& c, int kernel) {
  c.launches[kernel]++;
  // the class's precision: the nonlocal kernels follow the nonlocal term's (with kNlProj64 the
  // projections are float64 and add_vuspsi is not)
  const int np = nl_prec(c);
  bool at64;
  if (kernel == HPSI_K_CALBEC || kernel == HPSI_K_DSCALE) at64 = np == HPSI_FP64 || np == kNlProj64;
  else if (kernel == HPSI_K_ADDVUS) at64 = np == HPSI_FP64;
  else at64 = cur_prec(c) == HPSI_FP64;
  if (at64) c.launches64[kernel]++;
  if (!c.timing) return -1;
  cudaEvent_t a = pooled_event(c), b = pooled_event(c);
  cudaEventRecord(a, c.stream);
  c.trec.push_back({kernel + (at64 ? HPSI_K_AT_FP64 : 0), {a, b}});
  return (int)c.trec.size() - 1;
}

void launch_end(Context& c, int slot) {
  if (slot >= 0) cudaEventRecord(c.trec[slot].second.second, c.stream);
}

static int collect_timing(Context& c) {
  if (c.trec.empty()) return HPSI_OK;
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel timing");
  for (auto& r : c.trec) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.second.first, r.second.second) == cudaSuccess) {
      const int k = r.first % HPSI_K_AT_FP64;
      c.tacc[k] += ms;
      if (r.first >= HPSI_K_AT_FP64) c.tacc64[k] += ms;
    }
    c.evpool.push_back(r.second.first);
    c.evpool.push_back(r.second.second);
  }
  c.trec.clear();
  return HPSI_OK;
}

int check_device_error(Context& c) {
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
  if (!c.d_err) return HPSI_OK;
  int v = 0;
  e = cudaMemcpy(&v, c.d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "error word read");
  if (v != 0) {
    cudaMemset(c.d_err, 0, sizeof(int));
    return fail(c, HPSI_ETIMEOUT, "a bounded device-side wait expired; the output of that call is invalid");
  }
  return HPSI_OK;
}

int ensure_buffer(Context& c, void** ptr, size_t* have, size_t need) {
  if (need <= *have && *ptr) return HPSI_OK;
  c.ws.epoch++;
  if (*ptr) {
    cudaStreamSynchronize(c.stream);
    cudaFree(*ptr);
    *ptr = nullptr;
    *have = 0;
  }
  cudaError_t e = cudaMalloc(ptr, std::max<size_t>(need, 256));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(c, HPSI_ENOMEM, "device allocation of " + std::to_string(need) + " bytes failed");
  }
  *have = std::max<size_t>(need, 256);
  return HPSI_OK;
}

// <k+G|H|k+G> = |k+G|^2/2 + mean(V) + sum_{(p,q) in D} Re(beta_p(G) D_pq conj(beta_q(G)))
__global__ void k_hdiag(int npw, double vmean, const double* __restrict__ kin, const double2* __restrict__ beta,
                        int nproj, const int* __restrict__ rowptr, const int* __restrict__ col,
                        const double2* __restrict__ val, double* __restrict__ out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npw) return;
  double acc = kin[g] + vmean;
  for (int p = 0; p < nproj; ++p) {
    const double2 bp = beta[(size_t)p * npw + g];
    for (int e = rowptr[p]; e < rowptr[p + 1]; ++e) {
      const double2 bq = beta[(size_t)col[e] * npw + g];
      const double2 d = val[e];
      // Re( bp * d * conj(bq) )
      const double tx = bp.x * d.x - bp.y * d.y, ty = bp.x * d.y + bp.y * d.x;
      acc += tx * bq.x + ty * bq.y;
    }
  }
  out[g] = acc;
}

template <typename T>
static int upload(Context& c, T** dst, const T* src, size_t n) {
  if (n == 0) {
    *dst = nullptr;
    return HPSI_OK;
  }
  cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HPSI_ENOMEM, "device allocation failed during setup");
  }
  e = cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "setup upload");
  // the host source may be freed by the caller right after setup returns
  e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "setup upload");
  return HPSI_OK;
}

static int init_device(Context& c, void* stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetDeviceProperties");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(c, HPSI_ENODEV, std::string("libhpsi is built for sm_103a (GB300); device is ") + prop.name);
  c.device = dev;
  c.sm_count = prop.multiProcessorCount;
  c.smem_optin = prop.sharedMemPerBlockOptin;
  c.stream = reinterpret_cast<cudaStream_t>(stream);
  return HPSI_OK;
}

// V[j1][j2][j3] (host, C order) -> device V[j3][j2][j1] in float64 and float32; returns slot.
static int upload_potential(Context& c, const int n[3], const double* vr, int* slot, double* vmean) {
  const size_t nr = (size_t)n[0] * n[1] * n[2];
  std::vector<double> t(nr);
  std::vector<float> t32(nr);
  double s = 0.0;
  for (int j1 = 0; j1 < n[0]; ++j1)
    for (int j2 = 0; j2 < n[1]; ++j2)
      for (int j3 = 0; j3 < n[2]; ++j3) {
        const double v = vr[((size_t)j1 * n[1] + j2) * n[2] + j3];
        if (!std::isfinite(v)) return fail(c, HPSI_EINVAL, "vloc_r contains a non-finite value");
        s += v;
        const size_t o = ((size_t)j3 * n[1] + j2) * n[0] + j1;
        t[o] = v;
        t32[o] = (float)v;
      }
  *vmean = s / (double)nr;
  double* d64 = nullptr;
  float* d32 = nullptr;
  int rc = upload(c, &d64, t.data(), nr);
  if (rc) return rc;
  c.vbufs.push_back(d64);
  rc = upload(c, &d32, t32.data(), nr);
  if (rc) return rc;
  c.vbufs.push_back(d32);
  *slot = (int)c.vbufs.size() - 2;
  return HPSI_OK;
}

static int plan_for(Context& c, int n, FftPlan* out) {
  for (auto& t : c.tw)
    if (t.n == n) {
      *out = t.plan;
      return HPSI_OK;
    }
  TwiddleTable tt;
  tt.n = n;
  std::vector<double2> tab;
  make_fft_plan(n, tt.plan, tab);
  std::vector<float2> tab32(tab.size());
  for (size_t i = 0; i < tab.size(); ++i) tab32[i] = make_float2((float)tab[i].x, (float)tab[i].y);
  int rc = upload(c, &tt.d64, tab.data(), tab.size());
  if (rc) return rc;
  rc = upload(c, &tt.d32, tab32.data(), tab32.size());
  if (rc) return rc;
  std::vector<double2> nat(n);
  std::vector<float2> nat32(n);
  for (int j = 0; j < n; ++j) {
    const double ang = -6.283185307179586476925286766559 * (double)j / (double)n;
    nat[j] = make_double2(std::cos(ang), std::sin(ang));
    nat32[j] = make_float2((float)nat[j].x, (float)nat[j].y);
  }
  rc = upload(c, &tt.nat64, nat.data(), nat.size());
  if (rc) return rc;
  rc = upload(c, &tt.nat32, nat32.data(), nat32.size());
  if (rc) return rc;
  tt.plan.tw64 = tt.d64;
  tt.plan.tw32 = tt.d32;
  c.tw.push_back(tt);
  *out = tt.plan;
  return HPSI_OK;
}

// Whether the Gamma-point real form (Sec. 4) applies to a problem: k = 0, entry npw-1-i of the
// sphere's order is -G of entry i, and H maps real functions to real ones.  V is real, so that
// comes down to the projectors: beta_p(-G) = u_p conj(beta_p(G)) for every G with one |u_p| = 1
// per projector, and conj(u_p) u_q conj(D_pq) = D_pq for the nonzeros of D (then the nonlocal
// kernel K(G, G') satisfies conj(K(-G, -G')) = K(G, G')).  Checked to 1e-12 relative.
static bool gamma_applies(Problem& p, const double* beta, const double* dmat, std::string* why) {
  if (p.k[0] != 0.0 || p.k[1] != 0.0 || p.k[2] != 0.0) {
    *why = "the problem is not at k = 0";
    return false;
  }
  const int n = p.npw;
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a)
      if (p.miller[(size_t)(n - 1 - i) * 3 + a] != -p.miller[(size_t)i * 3 + a]) {
        *why = "the sphere is not symmetric under G -> -G";
        return false;
      }
  const int P = p.nproj;
  if (P == 0) return true;
  const double2* B = reinterpret_cast<const double2*>(beta);
  const double2* D = reinterpret_cast<const double2*>(dmat);
  std::vector<double2> u(P);
  for (int q = 0; q < P; ++q) {
    const double2* b = B + (size_t)q * n;
    int imax = 0;
    double amax = 0.0;
    for (int i = 0; i < n; ++i) {
      const double a = std::hypot(b[i].x, b[i].y);
      if (a > amax) {
        amax = a;
        imax = i;
      }
    }
    if (amax == 0.0) {
      u[q] = make_double2(1.0, 0.0);
      continue;
    }
    // u = beta(-G) / conj(beta(G)) at the largest component
    const double2 bp = b[imax], bm = b[n - 1 - imax];
    const double den = bp.x * bp.x + bp.y * bp.y;
    u[q] = make_double2((bm.x * bp.x - bm.y * bp.y) / den, (bm.x * bp.y + bm.y * bp.x) / den);
    const double tol = 1e-12 * amax;
    for (int i = 0; i < n; ++i) {
      const double2 x = b[i], y = b[n - 1 - i];
      const double rx = u[q].x * x.x + u[q].y * x.y, ry = u[q].y * x.x - u[q].x * x.y;   // u conj(x)
      if (std::fabs(y.x - rx) > tol || std::fabs(y.y - ry) > tol) {
        *why = "projector " + std::to_string(q) + " has no beta(-G) = u conj(beta(G)) symmetry";
        return false;
      }
    }
  }
  double dmax = 0.0;
  for (size_t i = 0; i < (size_t)P * P; ++i) dmax = std::max(dmax, std::hypot(D[i].x, D[i].y));
  for (int a = 0; a < P; ++a)
    for (int b = 0; b < P; ++b) {
      const double2 d = D[(size_t)a * P + b];
      if (d.x == 0.0 && d.y == 0.0) continue;
      // conj(u_a) u_b conj(d)
      const double2 w = make_double2(u[a].x * u[b].x + u[a].y * u[b].y, u[a].x * u[b].y - u[a].y * u[b].x);
      const double rx = w.x * d.x + w.y * d.y, ry = w.y * d.x - w.x * d.y;
      if (std::fabs(rx - d.x) > 1e-12 * dmax || std::fabs(ry - d.y) > 1e-12 * dmax) {
        *why = "D couples projectors whose phases make the nonlocal term complex";
        return false;
      }
    }
  p.gamma_u = u;
  return true;
}

__global__ void k_v_to_f32(size_t n, const double* __restrict__ v, float* __restrict__ v32) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    v32[i] = (float)v[i];
}

// Replace the local potential of problem ik (and of every problem sharing its V) by v64, a device
// float64 array [n3][n2][n1] with mean vmean; the diagonal <k+G|H|k+G> follows.
int set_potential(Context& c, int ik, const double* v64, double vmean) {
  Problem& p0 = c.probs[ik];
  const size_t nr = (size_t)p0.n[0] * p0.n[1] * p0.n[2];
  double* d64 = static_cast<double*>(c.vbufs[p0.vslot]);
  float* d32 = static_cast<float*>(c.vbufs[p0.vslot + 1]);
  cudaError_t e = cudaMemcpyAsync(d64, v64, sizeof(double) * nr, cudaMemcpyDeviceToDevice, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "potential update");
  HPSI_LAUNCH(c, HPSI_K_SCF, (k_v_to_f32<<<(int)std::min<size_t>(4096, (nr + 255) / 256), 256, 0, c.stream>>>(nr, d64, d32)));
  for (Problem& p : c.probs) {
    if (p.vslot != p0.vslot) continue;
    HPSI_LAUNCH(c, HPSI_K_SCF,
                (k_hdiag<<<(p.npw + 255) / 256, 256, 0, c.stream>>>(p.npw, vmean, p.d_kin, p.d_beta, p.nproj,
                                                                    p.d_rowptr, p.d_col, p.d_dval, p.d_hdiag)));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "potential update kernels");
  return HPSI_OK;
}

// Everything of one problem after its sphere is known: geometry, plans, device copies, D, hdiag.
static int finish_problem(Context& c, Problem& p, const double* vr, int vslot_shared, double vmean,
                          const double* beta, const double* dmat) {
  std::string err;
  int rc = build_geometry(p, err);
  if (rc) return fail(c, rc, err);
  for (int w = 0; w < 3; ++w)
    if (local_smem_bytes(p, HPSI_FP64, w) > c.smem_optin)
      return fail(c, HPSI_EINVAL, "FFT box / sphere too large for one CTA's shared memory");
  for (int a = 0; a < 3; ++a) {
    rc = plan_for(c, p.n[a], &p.plan[a]);
    if (rc) return rc;
  }
  if ((rc = upload(c, &p.d_sticks, p.sticks.data(), p.sticks.size()))) return rc;
  {
    // lookup maps of the fast path: stick of (plane, j2) and plane of ix
    std::vector<int> ymap((size_t)p.npl * p.n[1], -1), xmap(p.n[0], -1);
    for (int q = 0; q < p.npl; ++q) {
      xmap[p.planes[q].ix] = q;
      for (int s = p.planes[q].s0; s < p.planes[q].s0 + p.planes[q].ns; ++s)
        ymap[(size_t)q * p.n[1] + p.sticks[s].iy] = s;
    }
    if ((rc = upload(c, &p.d_ymap, ymap.data(), ymap.size()))) return rc;
    if ((rc = upload(c, &p.d_xmap, xmap.data(), xmap.size()))) return rc;
    for (auto& t : c.tw)
      if (t.n == p.n[0]) {
        p.d_ftw64 = t.nat64;
        p.d_ftw32 = t.nat32;
      }
    for (int pr = 0; pr < 2; ++pr) p.fflags[pr] = local_fast_plan(p, pr, c.smem_optin);
  }
  if ((rc = upload(c, &p.d_planes, p.planes.data(), p.planes.size()))) return rc;
  if ((rc = upload(c, &p.d_kin, p.kin.data(), p.kin.size()))) return rc;
  // the external (local pseudo)potential as given, in the device layout [n3][n2][n1], for the
  // self-consistency loop, which adds V_Hxc to it
  p.vext.resize((size_t)p.n[0] * p.n[1] * p.n[2]);
  for (int j1 = 0; j1 < p.n[0]; ++j1)
    for (int j2 = 0; j2 < p.n[1]; ++j2)
      for (int j3 = 0; j3 < p.n[2]; ++j3)
        p.vext[((size_t)j3 * p.n[1] + j2) * p.n[0] + j1] = vr[((size_t)j1 * p.n[1] + j2) * p.n[2] + j3];
  p.vslot = vslot_shared;
  p.d_v64 = reinterpret_cast<const double*>(c.vbufs[vslot_shared]);
  p.d_v32 = reinterpret_cast<const float*>(c.vbufs[vslot_shared + 1]);
  // projectors and D (CSR of its nonzeros)
  const int P = p.nproj;
  std::vector<int> rowptr(P + 1, 0), col;
  std::vector<double2> val;
  if (P > 0) {
    const double2* D = reinterpret_cast<const double2*>(dmat);
    double dmax = 0.0;
    for (int i = 0; i < P * P; ++i) dmax = std::max(dmax, std::hypot(D[i].x, D[i].y));
    for (int i = 0; i < P; ++i) {
      for (int j = 0; j < P; ++j) {
        const double2 a = D[(size_t)i * P + j], b = D[(size_t)j * P + i];
        if (!std::isfinite(a.x) || !std::isfinite(a.y)) return fail(c, HPSI_EINVAL, "dmat contains a non-finite value");
        if (std::fabs(a.x - b.x) > 1e-12 * dmax + 1e-300 || std::fabs(a.y + b.y) > 1e-12 * dmax + 1e-300)
          return fail(c, HPSI_EINVAL, "dmat is not Hermitian");
        if (a.x != 0.0 || a.y != 0.0) {
          col.push_back(j);
          val.push_back(a);
        }
      }
      rowptr[i + 1] = (int)col.size();
    }
    p.nnz = (int)col.size();
    const double2* B = reinterpret_cast<const double2*>(beta);
    for (size_t i = 0; i < (size_t)P * p.npw; ++i)
      if (!std::isfinite(B[i].x) || !std::isfinite(B[i].y)) return fail(c, HPSI_EINVAL, "beta contains a non-finite value");
    if ((rc = upload(c, &p.d_beta, B, (size_t)P * p.npw))) return rc;
    if ((rc = upload(c, &p.d_rowptr, rowptr.data(), rowptr.size()))) return rc;
    if (p.nnz) {
      if ((rc = upload(c, &p.d_col, col.data(), col.size()))) return rc;
      if ((rc = upload(c, &p.d_dval, val.data(), val.size()))) return rc;
    }
  } else {
    if ((rc = upload(c, &p.d_rowptr, rowptr.data(), rowptr.size()))) return rc;
  }
  p.gamma_ok = gamma_applies(p, beta, dmat, &p.gamma_why);
  cudaError_t e = cudaMalloc((void**)&p.d_hdiag, sizeof(double) * std::max(1, p.npw));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HPSI_ENOMEM, "device allocation failed during setup");
  }
  HPSI_LAUNCH(c, HPSI_K_DAVIDSON,
              (k_hdiag<<<(p.npw + 255) / 256, 256, 0, c.stream>>>(p.npw, vmean, p.d_kin, p.d_beta, P, p.d_rowptr,
                                                                  p.d_col, p.d_dval, p.d_hdiag)));
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "hdiag kernel");
  // band blocks of the local kernels: one block's intermediates stay near 48 MB (L2-resident)
  for (int pr = 0; pr < 2; ++pr) {
    const size_t cs = pr == HPSI_FP64 ? 16 : 8;
    const size_t xper = cs * (size_t)p.n[2] * p.npl * p.n[1];
    p.nbb[pr] = (int)std::max<size_t>(1, std::min<size_t>(4096, (size_t)(48u << 20) / std::max<size_t>(1, xper)));
    const size_t zper = 2 * cs * (size_t)p.n[2] * p.nst;
    p.nbbf[pr] = (int)std::max<size_t>(1, std::min<size_t>(4096, (size_t)(48u << 20) / std::max<size_t>(1, zper)));
  }
  if (c.precision == HPSI_MIXED && P > 0) {
    rc = mixed_prepare_beta(c, p);
    if (rc) return rc;
  }
  e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "setup");
  return HPSI_OK;
}

static void free_problem(Problem& p) {
  cudaFree(p.d_sticks);
  cudaFree(p.d_planes);
  cudaFree(p.d_ymap);
  cudaFree(p.d_xmap);
  cudaFree(p.d_kin);
  cudaFree(p.d_hdiag);
  cudaFree(p.d_beta);
  cudaFree(p.d_rowptr);
  cudaFree(p.d_col);
  cudaFree(p.d_dval);
  cudaFree(p.d_beta_bf);
  cudaFree(p.d_betar);
  cudaFree(p.d_dvalr);
  cudaFree(p.d_betar_bf);
  cudaFree(p.d_betar_df);
}

static void free_context(Context& c) {
  cudaStreamSynchronize(c.stream);
  collect_timing(c);
  for (cudaEvent_t e : c.evpool) cudaEventDestroy(e);
  c.evpool.clear();
  for (auto& p : c.probs) free_problem(p);
  for (auto& t : c.tw) {
    cudaFree(t.d64);
    cudaFree(t.d32);
    cudaFree(t.nat64);
    cudaFree(t.nat32);
  }
  for (void* v : c.vbufs) cudaFree(v);
  cudaFree(c.d_err);
  cudaFree(c.ws.X);
  cudaFree(c.ws.Y);
  cudaFree(c.ws.part);
  cudaFree(c.ws.w);
  cudaFree(c.ws.stage_in);
  cudaFree(c.ws.stage_out);
  cudaFree(c.ws.mixed);
  cudaFree(c.ws.batch);
  cudaFree(c.ws.gin);
  cudaFree(c.ws.gout);
  cudaFree(c.ws.gnl);
  cudaFree(c.ws.gdf);
  if (c.graph.exec) cudaGraphExecDestroy(c.graph.exec);
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  davidson_release(c);
  eigh_release(c);
  cg_release(c);
  gamma_release(c);
  scf_release(c);
  fock_release(c);
}

int nonlocal_apply(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd) {
  const int np = nl_prec(c);
  if (np == HPSI_FP64 || (np == kNlProj64 && c.precision != HPSI_MIXED))
    return nonlocal_apply_fp64(c, p, psi, hpsi, nbnd);
  if (np == kNlProj64) {
    if (p.nproj == 0 || nbnd == 0) return HPSI_OK;
    double2* w = nullptr;
    const int rc = nonlocal_w_fp64(c, p, psi, nbnd, &w);
    if (rc) return rc;
    return nonlocal_add_tc(c, p, w, hpsi, nbnd);
  }
  return nonlocal_apply_mixed(c, p, psi, hpsi, nbnd);
}

int apply_device(Context& c, int ik, const double2* psi, double2* hpsi, int nbnd) {
  const Problem& p = c.probs[ik];
  c.band_apps += nbnd;
  int rc = local_apply(c, p, psi, hpsi, nbnd);
  if (rc) return rc;
  return nonlocal_apply(c, p, psi, hpsi, nbnd);
}

// All items at once.  Problems whose box has the fast kernels share, per box edge, one persistent
// cooperative launch (the three FFT phases and, when the nonlocal term is float64, its three phases
// too), or, with HPSI_OPT_PERSISTENT off or when another item takes the generic path, one launch per
// kernel and box edge; their stick rows live side by side in one workspace.  The tensor-core
// nonlocal term follows per item.
static int batch_apply_items(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                             double2* const* hpsi) {
  std::vector<int> fast, slow;
  for (int i = 0; i < nitem; ++i) {
    if (nbnd[i] == 0) continue;
    const Problem& p = c.probs[prob[i]];
    if ((p.fflags[cur_prec(c)] & 4) && !c.force_generic) fast.push_back(i);
    else slow.push_back(i);
  }
  std::stable_sort(fast.begin(), fast.end(),
                   [&](int x, int y) { return c.probs[prob[x]].n[0] < c.probs[prob[y]].n[0]; });
  const size_t cs = cur_prec(c) == HPSI_FP64 ? sizeof(double2) : sizeof(float2);
  std::vector<size_t> off(fast.size());
  size_t total = 0;
  for (size_t j = 0; j < fast.size(); ++j) {
    const Problem& p = c.probs[prob[fast[j]]];
    off[j] = total;
    total += 2 * ((cs * (size_t)nbnd[fast[j]] * p.n[2] * p.nst + 255) & ~size_t(255));
  }
  if (!fast.empty()) {
    int rc = ensure_buffer(c, &c.ws.batch, &c.ws.batchbytes, total);
    if (rc) return rc;
    std::vector<int> fp(fast.size()), fn(fast.size());
    std::vector<const double2*> fi(fast.size());
    std::vector<double2*> fo(fast.size());
    std::vector<void*> zt(fast.size()), yb(fast.size());
    unsigned char* base = static_cast<unsigned char*>(c.ws.batch);
    for (size_t j = 0; j < fast.size(); ++j) {
      const int i = fast[j];
      const Problem& p = c.probs[prob[i]];
      fp[j] = prob[i];
      fn[j] = nbnd[i];
      fi[j] = psi[i];
      fo[j] = hpsi[i];
      zt[j] = base + off[j];
      yb[j] = base + off[j] + ((cs * (size_t)nbnd[i] * p.n[2] * p.nst + 255) & ~size_t(255));
    }
    // one persistent launch per box edge (up to 32 items each), with the float64 nonlocal term of
    // its items; a group whose launch does not fit takes the launch-per-kernel path
    if (c.persistent && slow.empty()) {
      const bool with_nl = nl_prec(c) == HPSI_FP64;
      const int nf = (int)fast.size();
      for (int g0 = 0; g0 < nf;) {
        const Problem& q = c.probs[fp[g0]];
        int g1 = g0 + 1;
        while (g1 < nf && g1 - g0 < 32 && c.probs[fp[g1]].n[0] == q.n[0]) ++g1;
        const int n = g1 - g0;
        bool done = false;
        rc = local_batch_persistent(c, n, fp.data() + g0, fn.data() + g0, fi.data() + g0, fo.data() + g0,
                                    zt.data() + g0, yb.data() + g0, with_nl, &done);
        if (rc) return rc;
        if (!done) {
          rc = local_fast_apply_multi(c, n, fp.data() + g0, fn.data() + g0, fi.data() + g0, fo.data() + g0,
                                      zt.data() + g0, yb.data() + g0);
          if (rc) return rc;
          if (with_nl) {
            rc = nonlocal_batch_fp64(c, n, fp.data() + g0, fn.data() + g0, fi.data() + g0, fo.data() + g0);
            if (rc) return rc;
          }
        }
        g0 = g1;
      }
      for (int i = 0; i < nitem; ++i) {
        if (nbnd[i] == 0) continue;
        if (!with_nl) {
          rc = nonlocal_apply(c, c.probs[prob[i]], psi[i], hpsi[i], nbnd[i]);
          if (rc) return rc;
        }
        c.band_apps += nbnd[i];
      }
      return HPSI_OK;
    }
    rc = local_fast_apply_multi(c, (int)fast.size(), fp.data(), fn.data(), fi.data(), fo.data(), zt.data(), yb.data());
    if (rc) return rc;
  }
  for (int i : slow) {
    int rc = local_apply(c, c.probs[prob[i]], psi[i], hpsi[i], nbnd[i]);
    if (rc) return rc;
  }
  // the nonlocal term: in float64 all items share one launch per kernel class; the tensor-core
  // form runs per item
  if (nl_prec(c) == HPSI_FP64) {
    int rc = nonlocal_batch_fp64(c, nitem, prob, nbnd, psi, hpsi);
    if (rc) return rc;
  }
  for (int i = 0; i < nitem; ++i) {
    if (nbnd[i] == 0) continue;
    if (nl_prec(c) != HPSI_FP64) {
      int rc = nonlocal_apply(c, c.probs[prob[i]], psi[i], hpsi[i], nbnd[i]);
      if (rc) return rc;
    }
    c.band_apps += nbnd[i];
  }
  return HPSI_OK;
}

// 1 = device (or managed), 0 = host, -1 = error
int pointer_kind(const void* ptr) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return 1;
  return 0;
}

// In a mixed context, whether the batch's nonlocal term runs in float64 on the CUDA cores, one launch
// per kernel class over all items (HPSI_OPT_BATCH_NL): the tensor-core form works on tiles of 128
// projector rows, and with a few projectors per item its per-item launches are mostly empty tiles.
static bool batch_nl64(const Context& c, int nitem, const int* prob, const int* nbnd) {
  if (c.precision != HPSI_MIXED || nl_prec(c) != HPSI_MIXED || c.batch_nl == 1) return false;
  if (c.batch_nl == 2) return true;
  for (int i = 0; i < nitem; ++i)
    if (nbnd[i] > 0 && c.probs[prob[i]].nproj > kBatchNl64MaxProj) return false;
  return true;
}

int batch_apply(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                double2* const* hpsi) {
  if (!batch_nl64(c, nitem, prob, nbnd)) return batch_apply_items(c, nitem, prob, nbnd, psi, hpsi);
  const int saved = c.nl_prec_override;
  c.nl_prec_override = HPSI_FP64;
  const int rc = batch_apply_items(c, nitem, prob, nbnd, psi, hpsi);
  c.nl_prec_override = saved;
  return rc;
}

}  // namespace hpsi

using namespace hpsi;

static bool check_cell(const double* cell) {
  if (!cell) return false;
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(cell[i])) return false;
  return true;
}

extern "C" int hpsi_gsphere(const double cell[9], double ecut, const double k_cart[3], int* npw_out,
                            int32_t* miller_out, int capacity) {
  if (!check_cell(cell) || !k_cart || !npw_out) {
    g_setup_err = "hpsi_gsphere: null or non-finite argument";
    return HPSI_EINVAL;
  }
  std::vector<int32_t> m;
  std::string err;
  int rc = enumerate_gsphere(cell, ecut, k_cart, m, err);
  if (rc) {
    g_setup_err = err;
    return rc;
  }
  const int npw = (int)(m.size() / 3);
  *npw_out = npw;
  if (miller_out) {
    if (capacity < npw) {
      g_setup_err = "hpsi_gsphere: capacity smaller than npw";
      return HPSI_EINVAL;
    }
    std::memcpy(miller_out, m.data(), m.size() * sizeof(int32_t));
  }
  return HPSI_OK;
}

static int setup_common(hpsi_ctx** out, int precision, void* stream, hpsi_ctx** ctx_out) {
  if (!out) {
    g_setup_err = "out is NULL";
    return HPSI_EINVAL;
  }
  *out = nullptr;
  if (precision != HPSI_FP64 && precision != HPSI_MIXED) {
    g_setup_err = "precision must be HPSI_FP64 or HPSI_MIXED";
    return HPSI_EINVAL;
  }
  hpsi_ctx* h = new (std::nothrow) hpsi_ctx();
  if (!h) {
    g_setup_err = "host allocation failed";
    return HPSI_ENOMEM;
  }
  h->c.precision = precision;
  int rc = init_device(h->c, stream);
  if (rc == HPSI_OK) {
    if (cudaMalloc((void**)&h->c.d_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(h->c.d_err, 0, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      h->c.err = "device allocation of the error word failed";
      rc = HPSI_ENOMEM;
    }
  }
  if (rc) {
    g_setup_err = h->c.err;
    cudaFree(h->c.d_err);
    delete h;
    return rc;
  }
  *ctx_out = h;
  return HPSI_OK;
}

static int setup_fail(hpsi_ctx* h, int rc) {
  g_setup_err = h->c.err;
  free_context(h->c);
  delete h;
  return rc;
}

extern "C" int hpsi_setup(hpsi_ctx** out, const double cell[9], double ecut, int nk, const double* kpts,
                          const int fft[3], const double* vloc_r, int nproj, const double* beta,
                          const double* dmat, int precision, void* cuda_stream) {
  hpsi_ctx* h = nullptr;
  int rc = setup_common(out, precision, cuda_stream, &h);
  if (rc) return rc;
  Context& c = h->c;
  if (!check_cell(cell) || nk < 1 || !kpts || !fft || !vloc_r || nproj < 0 || (nproj > 0 && (!beta || !dmat))) {
    c.err = "hpsi_setup: bad argument (null pointer, nk < 1 or nproj < 0)";
    return setup_fail(h, HPSI_EINVAL);
  }
  for (int a = 0; a < 3; ++a)
    if (!fft_size_ok(fft[a])) {
      c.err = "FFT edge " + std::to_string(fft[a]) + " is not a 2*3*5-smooth integer in [8, 256]";
      return setup_fail(h, HPSI_EINVAL);
    }
  int slot = 0;
  double vmean = 0.0;
  rc = upload_potential(c, fft, vloc_r, &slot, &vmean);
  if (rc) return setup_fail(h, rc);
  size_t boff = 0;
  c.probs.resize(nk);
  for (int ik = 0; ik < nk; ++ik) {
    Problem& p = c.probs[ik];
    std::memcpy(p.cell, cell, sizeof(p.cell));
    reciprocal(p.cell, p.recip);
    p.ecut = ecut;
    for (int a = 0; a < 3; ++a) {
      p.k[a] = kpts[3 * ik + a];
      p.n[a] = fft[a];
      if (!std::isfinite(p.k[a])) {
        c.err = "non-finite k-point";
        return setup_fail(h, HPSI_EINVAL);
      }
    }
    std::string err;
    rc = enumerate_gsphere(p.cell, ecut, p.k, p.miller, err);
    if (rc) {
      c.err = err;
      return setup_fail(h, rc);
    }
    p.nproj = nproj;
    const double* bk = nproj > 0 ? beta + 2 * boff : nullptr;
    boff += (size_t)nproj * (p.miller.size() / 3);
    rc = finish_problem(c, p, vloc_r, slot, vmean, bk, dmat);
    if (rc) return setup_fail(h, rc);
  }
  *out = h;
  return HPSI_OK;
}

extern "C" int hpsi_setup_cells(hpsi_ctx** out, int ncell, const double* cells, const double* ecut, const int* fft,
                                const double* const* vloc_r, const int* nproj, const double* const* beta,
                                const double* const* dmat, int precision, void* cuda_stream) {
  hpsi_ctx* h = nullptr;
  int rc = setup_common(out, precision, cuda_stream, &h);
  if (rc) return rc;
  Context& c = h->c;
  if (ncell < 1 || !cells || !ecut || !fft || !vloc_r || !nproj) {
    c.err = "hpsi_setup_cells: bad argument";
    return setup_fail(h, HPSI_EINVAL);
  }
  c.probs.resize(ncell);
  for (int ic = 0; ic < ncell; ++ic) {
    Problem& p = c.probs[ic];
    if (!check_cell(cells + 9 * ic) || !vloc_r[ic] || nproj[ic] < 0 ||
        (nproj[ic] > 0 && (!beta || !dmat || !beta[ic] || !dmat[ic]))) {
      c.err = "hpsi_setup_cells: bad argument for cell " + std::to_string(ic);
      return setup_fail(h, HPSI_EINVAL);
    }
    std::memcpy(p.cell, cells + 9 * ic, sizeof(p.cell));
    reciprocal(p.cell, p.recip);
    p.ecut = ecut[ic];
    for (int a = 0; a < 3; ++a) {
      p.k[a] = 0.0;
      p.n[a] = fft[3 * ic + a];
      if (!fft_size_ok(p.n[a])) {
        c.err = "FFT edge " + std::to_string(p.n[a]) + " of cell " + std::to_string(ic) + " is not supported";
        return setup_fail(h, HPSI_EINVAL);
      }
    }
    int slot = 0;
    double vmean = 0.0;
    rc = upload_potential(c, p.n, vloc_r[ic], &slot, &vmean);
    if (rc) return setup_fail(h, rc);
    std::string err;
    rc = enumerate_gsphere(p.cell, p.ecut, p.k, p.miller, err);
    if (rc) {
      c.err = err;
      return setup_fail(h, rc);
    }
    p.nproj = nproj[ic];
    rc = finish_problem(c, p, vloc_r[ic], slot, vmean, p.nproj ? beta[ic] : nullptr, p.nproj ? dmat[ic] : nullptr);
    if (rc) return setup_fail(h, rc);
  }
  *out = h;
  return HPSI_OK;
}

extern "C" int hpsi_nprob(const hpsi_ctx* ctx) {
  if (!ctx) return HPSI_EINVAL;
  return (int)ctx->c.probs.size();
}

extern "C" int hpsi_npw(const hpsi_ctx* ctx, int ik) {
  if (!ctx || ik < 0 || ik >= (int)ctx->c.probs.size()) return HPSI_EINVAL;
  return ctx->c.probs[ik].npw;
}

extern "C" int hpsi_nproj(const hpsi_ctx* ctx, int ik) {
  if (!ctx || ik < 0 || ik >= (int)ctx->c.probs.size()) return HPSI_EINVAL;
  return ctx->c.probs[ik].nproj;
}

extern "C" int hpsi_apply(hpsi_ctx* ctx, int ik, const void* psi_in, void* hpsi_out, int nbnd) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  if (ik < 0 || ik >= (int)c.probs.size()) return fail(c, HPSI_EINVAL, "hpsi_apply: problem index out of range");
  if (nbnd < 0) return fail(c, HPSI_EINVAL, "hpsi_apply: nbnd < 0");
  if (nbnd == 0) return HPSI_OK;
  if (!psi_in || !hpsi_out) return fail(c, HPSI_EINVAL, "hpsi_apply: null pointer");
  const Problem& p = c.probs[ik];
  const size_t bytes = sizeof(double2) * (size_t)nbnd * p.npw;
  const char* a0 = static_cast<const char*>(psi_in);
  const char* b0 = static_cast<const char*>(hpsi_out);
  if (a0 < b0 + bytes && b0 < a0 + bytes) return fail(c, HPSI_EINVAL, "hpsi_apply: psi_in and hpsi_out overlap");
  const int ka = pointer_kind(psi_in), kb = pointer_kind(hpsi_out);
  if (ka < 0 || kb < 0 || ka != kb)
    return fail(c, HPSI_EINVAL, "hpsi_apply: psi_in and hpsi_out must both be device or both be host memory");
  if (ka == 1)
    return apply_device(c, ik, static_cast<const double2*>(psi_in), static_cast<double2*>(hpsi_out), nbnd);
  int rc = ensure_buffer(c, &c.ws.stage_in, &c.ws.stage_in_bytes, bytes);
  if (rc) return rc;
  rc = ensure_buffer(c, &c.ws.stage_out, &c.ws.stage_out_bytes, bytes);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(c.ws.stage_in, psi_in, bytes, cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "hpsi_apply host->device copy");
  rc = apply_device(c, ik, static_cast<const double2*>(c.ws.stage_in), static_cast<double2*>(c.ws.stage_out), nbnd);
  if (rc) return rc;
  e = cudaMemcpyAsync(hpsi_out, c.ws.stage_out, bytes, cudaMemcpyDeviceToHost, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "hpsi_apply device->host copy");
  return check_device_error(c);
}

extern "C" int hpsi_apply_batch(hpsi_ctx* ctx, int nitem, const int* prob, const int* nbnd,
                                const void* const* psi_in, void* const* hpsi_out) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  if (nitem < 0 || (nitem > 0 && (!prob || !nbnd || !psi_in || !hpsi_out)))
    return fail(c, HPSI_EINVAL, "hpsi_apply_batch: bad argument");
  for (int i = 0; i < nitem; ++i) {
    if (prob[i] < 0 || prob[i] >= (int)c.probs.size() || nbnd[i] < 0)
      return fail(c, HPSI_EINVAL, "hpsi_apply_batch: bad item " + std::to_string(i));
    if (nbnd[i] > 0 && (pointer_kind(psi_in[i]) != 1 || pointer_kind(hpsi_out[i]) != 1))
      return fail(c, HPSI_EINVAL, "hpsi_apply_batch: item pointers must be device memory");
  }
  std::vector<unsigned long long> key;
  key.push_back((unsigned long long)nitem);
  key.push_back((unsigned long long)(c.precision * 16 + c.nl_terms * 2 + c.force_generic));
  key.push_back((unsigned long long)(nl_prec(c) * 2 + (c.persistent ? 1 : 0) + 16 * c.batch_nl));
  for (int i = 0; i < nitem; ++i) {
    key.push_back((unsigned long long)prob[i]);
    key.push_back((unsigned long long)nbnd[i]);
    key.push_back((unsigned long long)reinterpret_cast<uintptr_t>(psi_in[i]));
    key.push_back((unsigned long long)reinterpret_cast<uintptr_t>(hpsi_out[i]));
  }
  const double2* const* pi = reinterpret_cast<const double2* const*>(psi_in);
  double2* const* po = reinterpret_cast<double2* const*>(hpsi_out);
  GraphCache& g = c.graph;
  if (g.exec && g.key == key && g.epoch == c.ws.epoch) {
    cudaError_t e = cudaGraphLaunch(g.exec, c.stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "hpsi_apply_batch graph launch");
    for (int k = 0; k < HPSI_K_COUNT; ++k) {
      c.launches[k] += g.launches[k];
      if (cur_prec(c) == HPSI_FP64) c.launches64[k] += g.launches[k];
    }
    c.band_apps += g.band_apps;
    return HPSI_OK;
  }
  // first call with these arguments: run it, then capture the same sequence for later calls
  long long before[HPSI_K_COUNT];
  for (int k = 0; k < HPSI_K_COUNT; ++k) before[k] = c.launches[k];
  const long long bapps0 = c.band_apps;
  int rc = batch_apply(c, nitem, prob, nbnd, pi, po);
  if (rc) return rc;
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  if (!c.cap_stream && cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return HPSI_OK;   // no capture stream: this call ran eagerly, later calls will too
  }
  long long after[HPSI_K_COUNT], after64[HPSI_K_COUNT];
  for (int k = 0; k < HPSI_K_COUNT; ++k) {
    after[k] = c.launches[k];
    after64[k] = c.launches64[k];
  }
  const long long bapps1 = c.band_apps;
  const long long epoch = c.ws.epoch;
  cudaStream_t orig = c.stream;
  const bool timing = c.timing;
  c.timing = false;
  c.stream = c.cap_stream;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal);
  int rc2 = e == cudaSuccess ? batch_apply(c, nitem, prob, nbnd, pi, po) : HPSI_ECUDA;
  cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(c.cap_stream, &graph) : e;
  c.stream = orig;
  c.timing = timing;
  for (int k = 0; k < HPSI_K_COUNT; ++k) {
    c.launches[k] = after[k];
    c.launches64[k] = after64[k];
  }
  c.band_apps = bapps1;
  if (rc2 == HPSI_OK && e2 == cudaSuccess && graph && c.ws.epoch == epoch) {
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
      g.exec = exec;
      g.key = key;
      g.epoch = epoch;
      for (int k = 0; k < HPSI_K_COUNT; ++k) g.launches[k] = after[k] - before[k];
      g.band_apps = bapps1 - bapps0;
    }
  }
  if (graph) cudaGraphDestroy(graph);
  cudaGetLastError();
  return HPSI_OK;
}

extern "C" int davidson_solve(hpsi_ctx* ctx, int ik, int nbnd, double tol, int maxiter, void* psi_inout,
                              double* eig_out, int* iters_out, double* resnorm_out) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  if (ik < 0 || ik >= (int)c.probs.size()) return fail(c, HPSI_EINVAL, "davidson_solve: problem index out of range");
  const Problem& p = c.probs[ik];
  if (nbnd < 1 || basis_of(c) * nbnd > p.npw)
    return fail(c, HPSI_EINVAL, "davidson_solve: need 1 <= nbnd and (basis factor) * nbnd <= npw");
  if (!(tol > 0.0) || maxiter < 1 || !psi_inout || !eig_out)
    return fail(c, HPSI_EINVAL, "davidson_solve: bad tol, maxiter or null pointer");
  const int kind = pointer_kind(psi_inout);
  if (kind < 0) return fail(c, HPSI_EINVAL, "davidson_solve: unrecognised psi pointer");
  const size_t bytes = sizeof(double2) * (size_t)nbnd * p.npw;
  if (kind == 1)
    return davidson_run(c, ik, nbnd, tol, maxiter, static_cast<double2*>(psi_inout), eig_out, iters_out, resnorm_out);
  int rc = ensure_buffer(c, &c.ws.stage_in, &c.ws.stage_in_bytes, bytes);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(c.ws.stage_in, psi_inout, bytes, cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "davidson_solve host->device copy");
  rc = davidson_run(c, ik, nbnd, tol, maxiter, static_cast<double2*>(c.ws.stage_in), eig_out, iters_out, resnorm_out);
  if (rc != HPSI_OK && rc != HPSI_ENOTCONV) return rc;
  e = cudaMemcpyAsync(psi_inout, c.ws.stage_in, bytes, cudaMemcpyDeviceToHost, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "davidson_solve device->host copy");
  e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "davidson_solve");
  return rc;
}

extern "C" int cg_solve(hpsi_ctx* ctx, int ik, int nbnd, double tol, int maxiter, void* psi_inout, double* eig_out,
                        int* iters_out, double* resnorm_out) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  if (ik < 0 || ik >= (int)c.probs.size()) return fail(c, HPSI_EINVAL, "cg_solve: problem index out of range");
  const Problem& p = c.probs[ik];
  if (nbnd < 1 || nbnd > p.npw) return fail(c, HPSI_EINVAL, "cg_solve: need 1 <= nbnd <= npw");
  if (!(tol > 0.0) || maxiter < 1 || !psi_inout || !eig_out)
    return fail(c, HPSI_EINVAL, "cg_solve: bad tol, maxiter or null pointer");
  const int kind = pointer_kind(psi_inout);
  if (kind < 0) return fail(c, HPSI_EINVAL, "cg_solve: unrecognised psi pointer");
  const size_t bytes = sizeof(double2) * (size_t)nbnd * p.npw;
  if (kind == 1) return cg_run(c, ik, nbnd, tol, maxiter, static_cast<double2*>(psi_inout), eig_out, iters_out, resnorm_out);
  int rc = ensure_buffer(c, &c.ws.stage_in, &c.ws.stage_in_bytes, bytes);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(c.ws.stage_in, psi_inout, bytes, cudaMemcpyHostToDevice, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cg_solve host->device copy");
  rc = cg_run(c, ik, nbnd, tol, maxiter, static_cast<double2*>(c.ws.stage_in), eig_out, iters_out, resnorm_out);
  if (rc != HPSI_OK && rc != HPSI_ENOTCONV) return rc;
  e = cudaMemcpyAsync(psi_inout, c.ws.stage_in, bytes, cudaMemcpyDeviceToHost, c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cg_solve device->host copy");
  e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cg_solve");
  return rc;
}

extern "C" int hpsi_set_option(hpsi_ctx* ctx, int option, double value) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  if (option == HPSI_OPT_PRECOND_TAU) {
    if (!(value > 0.0) || !std::isfinite(value)) return fail(c, HPSI_EINVAL, "HPSI_OPT_PRECOND_TAU must be > 0");
    c.opt_tau = value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_KERNEL_TIMING) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_KERNEL_TIMING must be 0 or 1");
    c.timing = value != 0.0;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_NL_TERMS) {
    if (value != 2.0 && value != 3.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_NL_TERMS must be 2 or 3");
    if ((int)value == c.nl_terms) return HPSI_OK;
    c.nl_terms = (int)value;
    if (c.precision == HPSI_MIXED) {
      cudaStreamSynchronize(c.stream);
      for (auto& p : c.probs) {
        if (p.nproj == 0) continue;
        cudaFree(p.d_beta_bf);
        p.d_beta_bf = nullptr;
        int rc = mixed_prepare_beta(c, p);
        if (rc) return rc;
      }
    }
    return HPSI_OK;
  }
  if (option == HPSI_OPT_FP32_GEMM) {
    if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0 && value != 4.0)
      return fail(c, HPSI_EINVAL, "HPSI_OPT_FP32_GEMM must be 0, 1, 2, 3 or 4");
    c.fp32_gemm = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_LOCKING) {
    if (value != 0.0 && value != 1.0 && value != 2.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_LOCKING must be 0, 1 or 2");
    c.locking = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_LOCK_BATCH) {
    if (!(value >= 0.0 && value <= 1.0)) return fail(c, HPSI_EINVAL, "HPSI_OPT_LOCK_BATCH must be in [0, 1]");
    c.lock_batch = value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_LOCK_BASIS) {
    if (!(value >= 2.0 && value <= 64.0) || value != std::floor(value))
      return fail(c, HPSI_EINVAL, "HPSI_OPT_LOCK_BASIS must be an integer in [2, 64]");
    c.lock_basis = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_THICK_RESTART) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_THICK_RESTART must be 0 or 1");
    c.thick_restart = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_CG_TMIN) {
    if (!(value > 0.0) || !std::isfinite(value)) return fail(c, HPSI_EINVAL, "HPSI_OPT_CG_TMIN must be > 0");
    c.cg_tmin = value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_SCF_NMIX) {
    if (!(value >= 1.0 && value <= 16.0) || value != std::floor(value))
      return fail(c, HPSI_EINVAL, "HPSI_OPT_SCF_NMIX must be an integer in [1, 16]");
    c.scf_nmix = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_SCF_BETA) {
    if (!(value > 0.0 && value <= 1.0)) return fail(c, HPSI_EINVAL, "HPSI_OPT_SCF_BETA must be in (0, 1]");
    c.scf_beta = value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_GAMMA_GEMM) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_GAMMA_GEMM must be 0 or 1");
    c.gamma_gemm = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_BATCH_NL) {
    if (value != 0.0 && value != 1.0 && value != 2.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_BATCH_NL must be 0, 1 or 2");
    c.batch_nl = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_PERSISTENT) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_PERSISTENT must be 0 or 1");
    c.persistent = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_EIGH_DF) {
    if (value != 0.0 && value != 1.0 && value != 2.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_EIGH_DF must be 0, 1 or 2");
    c.eigh_df = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_SCF_DAVIDSON_TOL) {
    if (!(value > 0.0) || !std::isfinite(value)) return fail(c, HPSI_EINVAL, "HPSI_OPT_SCF_DAVIDSON_TOL must be > 0");
    c.scf_dav_tol = value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_REORTH_TEST) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_REORTH_TEST must be 0 or 1");
    c.reorth_test = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_RITZ_SPLIT) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_RITZ_SPLIT must be 0 or 1");
    c.ritz_split = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_EIGENSOLVER) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_EIGENSOLVER must be 0 or 1");
    c.eigensolver = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_AUTOTUNE) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_AUTOTUNE must be 0 or 1");
    c.autotune = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_BASIS) {
    if (value != 0.0 && value != 2.0 && value != 3.0 && value != 4.0)
      return fail(c, HPSI_EINVAL, "HPSI_OPT_BASIS must be 0, 2, 3 or 4");
    c.basis_factor = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_FINAL_FP64) {
    if (value != 0.0 && value != 1.0 && value != 2.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_FINAL_FP64 must be 0, 1 or 2");
    c.final_fp64 = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_TC_KSPLIT) {
    if (!(value >= 0.0) || value > 1e6) return fail(c, HPSI_EINVAL, "HPSI_OPT_TC_KSPLIT must be >= 0");
    c.tc_kmax = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_LOCAL_PATH) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_LOCAL_PATH must be 0 or 1");
    c.force_generic = (int)value;
    return HPSI_OK;
  }
  if (option == HPSI_OPT_PRECOND_SHIFT) {
    if (value != 0.0 && value != 1.0) return fail(c, HPSI_EINVAL, "HPSI_OPT_PRECOND_SHIFT must be 0 or 1");
    c.opt_shift = (int)value;
    return HPSI_OK;
  }
  return fail(c, HPSI_EINVAL, "unknown option " + std::to_string(option));
}

extern "C" int hpsi_kernel_stats(hpsi_ctx* ctx, int kernel, long long* launches, double* total_ms, int reset) {
  if (!ctx) return HPSI_EINVAL;
  Context& c = ctx->c;
  const bool only64 = kernel >= HPSI_K_AT_FP64;
  if (only64) kernel -= HPSI_K_AT_FP64;
  if (kernel < -4 || kernel >= HPSI_K_COUNT || (only64 && kernel < 0))
    return fail(c, HPSI_EINVAL, "hpsi_kernel_stats: bad kernel class");
  if (kernel == -4) {
    if (launches) *launches = c.tri_calls;
    if (total_ms) *total_ms = c.tri_flops;
    if (reset) {
      c.tri_calls = 0;
      c.tri_flops = 0.0;
    }
    return HPSI_OK;
  }
  if (kernel == -3) {
    if (launches) *launches = c.eig_calls;
    if (total_ms) *total_ms = (double)c.eig_fallbacks;
    if (reset) c.eig_calls = c.eig_fallbacks = 0;
    return HPSI_OK;
  }
  if (kernel == -2) {
    if (launches) *launches = c.band_apps;
    if (total_ms) *total_ms = 0.0;
    if (reset) c.band_apps = 0;
    return HPSI_OK;
  }
  int rc = collect_timing(c);
  if (rc) return rc;
  long long n = 0;
  double ms = 0.0;
  for (int k = 0; k < HPSI_K_COUNT; ++k)
    if (kernel == -1 || kernel == k) {
      n += only64 ? c.launches64[k] : c.launches[k];
      if (kernel != -1) ms += only64 ? c.tacc64[k] : c.tacc[k];
    }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  if (reset)
    for (int k = 0; k < HPSI_K_COUNT; ++k)
      if (kernel == -1 || kernel == k) {
        c.launches[k] = c.launches64[k] = 0;
        c.tacc[k] = c.tacc64[k] = 0.0;
      }
  return HPSI_OK;
}

extern "C" int hpsi_selftest_timeout(hpsi_ctx* ctx) {
  if (!ctx) return HPSI_EINVAL;
  return wait_selftest(ctx->c);
}

extern "C" int hpsi_sync(hpsi_ctx* ctx) {
  if (!ctx) return HPSI_EINVAL;
  return check_device_error(ctx->c);
}

extern "C" const char* hpsi_last_error(const hpsi_ctx* ctx) {
  if (!ctx) return g_setup_err.c_str();
  return ctx->c.err.c_str();
}

extern "C" void hpsi_destroy(hpsi_ctx* ctx) {
  if (!ctx) return;
  free_context(ctx->c);
  delete ctx;
}
