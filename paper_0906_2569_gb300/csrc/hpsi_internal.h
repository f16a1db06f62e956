// Internal declarations of libhpsi: problem geometry, FFT plans, context, launchers.
#pragma once

#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hpsi.h"

namespace hpsi {

constexpr int kMaxFftN = 256;     // largest FFT edge supported by the warp FFT
constexpr int kMaxStages = 8;
constexpr int kWarpsPerCta = 8;   // local-potential kernels run 256 threads

// One radix pass list for a transform of length n (Stockham, radices 4, 2, 3, 5).
struct FftPlan {
  int n;
  int nstages;
  int radix[kMaxStages];
  int twoff[kMaxStages];   // offset of each stage's twiddles in the table of this n
  const double2* tw64;     // device: e^{-2 pi i r k / (Ns R)} for k < Ns, r = 1..R-1, per stage
  const float2* tw32;
};

// A z-column ("stick") of the sphere: G = (m1, m2, m3lo + t), t < len, stored at g0 + t.
struct StickDev {
  int g0;
  int len;
  int z0;   // m3lo mod n3
  int iy;   // m2 mod n2
};

// The sticks that share one m1 ("plane"): sticks s0 .. s0+ns-1, G's from g0.
struct PlaneDev {
  int s0;
  int ns;
  int ix;   // m1 mod n1
  int g0;
};

struct Problem {
  double cell[9];
  double recip[9];
  double ecut;
  double k[3];
  int n[3];
  int npw = 0, nst = 0, npl = 0, ns_max = 0, nproj = 0;
  std::vector<int32_t> miller;
  std::vector<StickDev> sticks;
  std::vector<PlaneDev> planes;
  std::vector<double> kin;      // |k+G|^2 / 2
  // device
  StickDev* d_sticks = nullptr;
  PlaneDev* d_planes = nullptr;
  double* d_kin = nullptr;
  double* d_hdiag = nullptr;
  const double* d_v64 = nullptr;   // V in [n3][n2][n1] layout (may be shared between problems)
  const float* d_v32 = nullptr;
  int vslot = -1;                  // index into Context::vbufs
  double2* d_beta = nullptr;
  int* d_rowptr = nullptr;
  int* d_col = nullptr;
  double2* d_dval = nullptr;
  int nnz = 0;
  uint16_t* d_beta_bf = nullptr;   // mixed path only
  FftPlan plan[3];
  // per precision (index HPSI_FP64 / HPSI_MIXED): band blocks and the fast-path plan
  int nbb[2] = {1, 1};             // band block of the generic local kernels
  mutable int fflags[2] = {0, 0};  // fast path: bit 2 enabled, bit 0 stage V, bit 1 stage the stick row
  mutable int nbbf[2] = {1, 1};    // band block of the fast local kernels
  mutable bool tuned[2] = {false, false};   // autotuner has chosen fflags / nbbf
  mutable int nl_kmax = 0;         // mixed calbec: K-steps per float32 accumulation the autotuner chose
                                   // (0: not tuned yet)
  int* d_ymap = nullptr;           // [npl][n2]: stick of (plane, j2) or -1
  int* d_xmap = nullptr;           // [n1]: plane of ix or -1
  const double2* d_ftw64 = nullptr;   // e^{-2 pi i j / n}, j < n (owned by the twiddle table)
  const float2* d_ftw32 = nullptr;
  std::vector<double> vext;        // the potential given at setup, host, layout [n3][n2][n1]
  bool gamma_ok = false;           // the Gamma-point real form applies (gamma.cu)
  std::string gamma_why;           // why not, when it does not
  std::vector<double2> gamma_u;    // per projector: beta(-G) = u conj(beta(G)) (when gamma_ok)
  // Gamma form, built on first use: the projectors rephased by conj(sqrt(u)) in real-basis
  // coordinates [P][2 nh], D in that basis (real, on D's CSR pattern), and (mixed contexts) their
  // bf16 terms: calbec's A [NT][P][round64(2 nh)], then add_vuspsi's B [NT][2 nh][round64(P)]
  double* d_betar = nullptr;
  double* d_dvalr = nullptr;
  uint16_t* d_betar_bf = nullptr;
  float2* d_betar_df = nullptr;    // (mixed contexts) betar as double-float pairs
};

struct TwiddleTable {
  int n;
  FftPlan plan;   // with device pointers filled
  double2* d64 = nullptr;
  float2* d32 = nullptr;
  double2* nat64 = nullptr;   // e^{-2 pi i j / n}, j < n
  float2* nat32 = nullptr;
};

struct Workspace {
  void* X = nullptr; size_t xbytes = 0;
  void* Y = nullptr; size_t ybytes = 0;
  void* part = nullptr; size_t partbytes = 0;    // split-K partials of <beta|psi>
  void* w = nullptr; size_t wbytes = 0;          // D <beta|psi>, [nb][P]
  void* stage_in = nullptr; size_t stage_in_bytes = 0;    // host-pointer staging
  void* stage_out = nullptr; size_t stage_out_bytes = 0;
  void* mixed = nullptr; size_t mixedbytes = 0;  // bf16 operand planes of the mixed path
  void* batch = nullptr; size_t batchbytes = 0;  // stick rows of a batched apply
  void* gin = nullptr; size_t ginbytes = 0;      // Gamma form: packed pairs of real bands, and H of them
  void* gout = nullptr; size_t goutbytes = 0;
  void* gnl = nullptr; size_t gnlbytes = 0;      // Gamma form: the float64 nonlocal term in real coordinates
  void* gdf = nullptr; size_t gdfbytes = 0;      // Gamma form: bands as double-float pairs
  void* pbar = nullptr; size_t pbarbytes = 0;    // grid-barrier counter of the persistent batch kernel
  long long epoch = 0;                           // bumped whenever a buffer is reallocated
};

// A captured hpsi_apply_batch sequence, replayed while its arguments and buffers are unchanged.
struct GraphCache {
  std::vector<unsigned long long> key;
  cudaGraphExec_t exec = nullptr;
  long long epoch = -1;
  long long launches[HPSI_K_COUNT] = {0};
  long long band_apps = 0;
};

struct Context {
  int precision = HPSI_FP64;
  cudaStream_t stream = nullptr;
  int device = 0;
  int sm_count = 152;
  size_t smem_optin = 0;
  std::vector<Problem> probs;
  std::vector<TwiddleTable> tw;
  std::vector<void*> vbufs;            // owned V buffers (64 and 32 bit)
  Workspace ws;
  std::string err;
  double opt_tau = 0.1;                // Davidson: |<k+G|H|k+G> - eps| is kept >= tau (Ha)
  int opt_shift = 0;                   // Davidson: 0 = eps_i per band, 1 = highest Ritz value
  void* blas = nullptr;                // Davidson handles and work buffers
  int* d_err = nullptr;                // device error word raised by bounded waits
  int nl_terms = 3;                    // mixed path: bf16 terms per operand (2 or 3)
  int force_generic = 0;               // 1: local part on the generic FFT kernels
  int tc_kmax = 0;                     // mixed calbec: max 64-wide K-steps per split (0: automatic)
  int prec_override = -1;              // >= 0: apply H at this precision instead of `precision`
  int nl_prec_override = -1;           // >= 0: the nonlocal term alone at this precision
  int final_fp64 = 2;                  // mixed davidson_solve: final Rayleigh quotients with float64
                                       // projections and D (2), the float64 H (1), the mixed H (0)
  int basis_factor = 0;                // Davidson: the reduced basis grows to basis_factor * N vectors
                                       // (0: 3 for a mixed context, 4 for float64)
  int autotune = 1;                    // time the fast-path plans on the first apply of a problem
  int persistent = 0;                  // hpsi_apply_batch: one persistent launch per box edge
  int batch_nl = 0;                    // hpsi_apply_batch, mixed: 0 auto, 1 tensor-core, 2 float64 batched
  int eigensolver = 1;                 // reduced eigenproblems: 1 = the library's kernels, 0 = cuSOLVER
  int fp32_gemm = 0;                   // mixed Davidson subspace GEMMs: 1 = bf16x9-emulated float32
  int locking = 0;                     // mixed Davidson: 0 none, 1 lowest converged run, 2 every converged band
  double lock_batch = 0.0;             // lock only once this fraction of the active bands is lockable
  int lock_basis = 4;                  // after a lock the active basis grows to lock_basis * active bands
  int thick_restart = 1;               // mixed Davidson: restarts keep up to half the basis limit of Ritz vectors
  int reorth_test = 0;                 // Davidson: second Gram-Schmidt pass only where the first cancelled
  int ritz_split = 0;                  // mixed Davidson: Ritz / restart GEMMs in K chunks added in float64
  void* eigh = nullptr;                // eigensolver handles and work buffers (eigh.cu)
  void* cg = nullptr;                  // conjugate-gradient solver handles and work buffers (cg.cu)
  void* gam = nullptr;                 // Gamma-point Davidson handles and work buffers (gamma.cu)
  void* scf = nullptr;                 // self-consistency loop buffers (scf.cu)
  void* fock = nullptr;                // exchange-operator buffers (fock.cu)
  int scf_nmix = 8;                    // SCF: past (input, residual) pairs the mixing combines
  double scf_beta = 0.5;               // SCF: step along the optimal residual
  double scf_dav_tol = 1e-9;           // SCF: residual tolerance of each Davidson solve
  int gamma_gemm = 1;                  // mixed Gamma Davidson: 1 bf16x9-emulated float32 GEMMs, 0 plain float32
  int eigh_df = 1;                     // real reduced problems: 0 float64; 1 double-float reduction and float32
                                       // eigenvector GEMMs in the mixed Gamma Davidson; 2 also the double-float
                                       // reduction in hpsi_eigh_lowest_sym and the float64 Gamma Davidson
  double cg_tmin = 1.0;                // CG preconditioner: P^2 = 1 / max(|k+G|^2/2, cg_tmin)
  cudaStream_t cap_stream = nullptr;   // internal stream for graph capture
  GraphCache graph;
  // launch accounting (always) and per-launch event timing (HPSI_OPT_KERNEL_TIMING)
  bool timing = false;
  long long launches[HPSI_K_COUNT] = {0};
  long long band_apps = 0;             // H|psi> band-applications performed
  long long eig_calls = 0;             // reduced eigenproblems solved by the library's kernels
  long long eig_fallbacks = 0;         // ... and handed to cuSOLVER instead
  long long tri_calls = 0;             // tridiagonal reductions run by the library
  double tri_flops = 0.0;              // sum over them of 16 n^3 / 3 (complex Hermitian)
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> trec;   // (kernel, start, end)
  std::vector<cudaEvent_t> evpool;
  double tacc[HPSI_K_COUNT] = {0.0};
  long long launches64[HPSI_K_COUNT] = {0};   // the part of launches made while H was applied in float64
  double tacc64[HPSI_K_COUNT] = {0.0};
};

// Precision at which H is applied right now.
inline int cur_prec(const Context& c) { return c.prec_override >= 0 ? c.prec_override : c.precision; }
// Precision of the nonlocal term right now: HPSI_FP64, HPSI_MIXED, or kNlProj64 (the projections
// <beta|psi> and D in float64, add_vuspsi on the tensor cores; mixed contexts only).
constexpr int kNlProj64 = 2;
// hpsi_apply_batch in a mixed context: items with at most this many projectors take the float64
// CUDA-core nonlocal term over the whole batch (HPSI_OPT_BATCH_NL = 0)
constexpr int kBatchNl64MaxProj = 64;
inline int nl_prec(const Context& c) { return c.nl_prec_override >= 0 ? c.nl_prec_override : cur_prec(c); }
// Bracket the final Rayleigh quotients of a mixed solve: HPSI_OPT_FINAL_FP64 1 applies H in float64;
// 2 the projections in float64 and the rest at the working precision.
inline void final_precision_begin(Context& c) {
  if (c.final_fp64 == 1) c.prec_override = HPSI_FP64;
  else if (c.final_fp64 == 2) c.nl_prec_override = kNlProj64;
}
inline void final_precision_end(Context& c) {
  c.prec_override = -1;
  c.nl_prec_override = -1;
}

// Bracket one launch: call before (returns a record slot or -1) and after the launch.
int launch_begin(Context& c, int kernel);
void launch_end(Context& c, int slot);
#define HPSI_LAUNCH(ctx, kid, ...)                 \
  do {                                             \
    const int slot_ = ::hpsi::launch_begin(ctx, kid); \
    __VA_ARGS__;                                   \
    ::hpsi::launch_end(ctx, slot_);                \
  } while (0)

// ---- host helpers (plan.cpp) ----
void reciprocal(const double cell[9], double recip[9]);
int enumerate_gsphere(const double cell[9], double ecut, const double k[3], std::vector<int32_t>& miller,
                      std::string& err);
bool fft_size_ok(int n);
void make_fft_plan(int n, FftPlan& plan, std::vector<double2>& table);
int build_geometry(Problem& p, std::string& err);

// ---- launchers (local_kernels.cu, nonlocal_fp64.cu) ----
// Complex64 inner products C = A^H B on the tcgen05 tensor cores (nonlocal_tc.cu): three bf16 terms
// per float32 operand (exact), six products accumulated in float32 per K-split, splits summed in
// float64.  A rows [0, M) and B rows [0, nb) are complex64 vectors of npw elements (ld npw).  With
// cache_a the bf16 split of A's rows is kept across calls (for a basis that only grows; call
// invalidate() when its rows change; rows_cap sizes the cache).  The result goes to out64 (or, when
// out64 is null, out32), column-major with leading dimension ldo: element (i, b) at i + b ldo.
struct TcInner {
  void* terms = nullptr;      // cached bf16 split of A: 3 planes of caprows x kpad
  const void* base = nullptr;
  int caprows = 0, kpad = 0, valid = 0;
  void* ws = nullptr;         // per-call splits and float partials
  size_t wsbytes = 0;
  void invalidate() { valid = 0; }
  void release();
};
int tc_inner32(Context& c, TcInner& t, bool cache_a, int rows_cap, const float2* A, int M, const float2* B, int nb,
               int npw, double2* out64, float2* out32, int ldo);

// The Davidson basis factor in effect: HPSI_OPT_BASIS, or by precision when it is left at 0.
inline int basis_of(const Context& c) { return c.basis_factor ? c.basis_factor : (c.precision == HPSI_MIXED ? 3 : 4); }

size_t local_smem_bytes(const Problem& p, int precision, int which);
int local_apply(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd);
int nonlocal_apply_fp64(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd);
int nonlocal_apply_mixed(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd);
int mixed_prepare_beta(Context& c, Problem& p);
int wait_selftest(Context& c);
size_t local_scratch_per_band(const Problem& p, int precision);
int local_fast_plan(const Problem& p, int precision, size_t smem_optin);
std::vector<int> local_fast_candidates(const Problem& p, int precision, size_t smem_optin);
int local_fast_apply(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, void* Zt, void* Yb,
                     int nbb);
int local_fast_apply_multi(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                           double2* const* hpsi, void* const* zt, void* const* yb);
// The whole batch (and with_nl its float64 nonlocal term) in one persistent cooperative launch;
// *done = false when it does not apply (the caller then launches per kernel class).
int local_batch_persistent(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                           double2* const* hpsi, void* const* zt, void* const* yb, bool with_nl, bool* done);
int nonlocal_apply(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd);
// rho[j3][j2][j1] += sum_b wb[b] |psi_b(r_j)|^2 (float64 bands, wb on the device; local_kernels.cu)
int local_density(Context& c, const Problem& p, const double2* psi, int nbnd, const double* wb, double* rho);
// Replace V of problem ik (and of the problems sharing it) by a device float64 [n3][n2][n1] array
int set_potential(Context& c, int ik, const double* v64, double vmean);
int batch_apply(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                double2* const* hpsi);
int local_apply_into(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, void* X, void* Y,
                     int nbb);
void nonlocal_fp64_plan(const Context& c, const Problem& p, int nbnd, int* nsplit, int* kchunk, size_t* bytes,
                        size_t max_bytes = 0);
int nonlocal_fp64_into(Context& c, const Problem& p, const double2* psi, double2* hpsi, int nbnd, void* scratch,
                       size_t capacity);
// The float64 nonlocal term of several problems' band blocks, one launch per kernel class
int nonlocal_batch_fp64(Context& c, int nitem, const int* prob, const int* nbnd, const double2* const* psi,
                        double2* const* hpsi);

// ---- context helpers (api.cpp) ----
int ensure_buffer(Context& c, void** ptr, size_t* have, size_t need);
int fail(Context& c, int code, const std::string& msg);
int cuda_fail(Context& c, cudaError_t e, const char* what);
int apply_device(Context& c, int ik, const double2* psi, double2* hpsi, int nbnd);
int check_device_error(Context& c);   // synchronizes; HPSI_ETIMEOUT if a bounded wait expired
int pointer_kind(const void* ptr);    // 1 device (or managed), 0 host, -1 unknown

// ---- Davidson (davidson.cu) ----
int davidson_run(Context& c, int ik, int nbnd, double tol, int maxiter, double2* psi, double* eig,
                 int* iters, double* resnorm);
void davidson_release(Context& c);
// Band-by-band preconditioned CG eigensolver of App. A.2.2 (cg.cu); psi on the device.
int cg_run(Context& c, int ik, int nbnd, double tol, int maxiter, double2* psi, double* eig, int* iters,
           double* resnorm);
void cg_release(Context& c);
// Gamma-point real form (gamma.cu): H on half-sphere bands (scaled: real-basis coordinates), block
// Davidson on real orbitals, and the check that a problem allows the form.
int gamma_apply(Context& c, int ik, const double2* x, double2* y, int nb, bool scaled);
int gamma_check(Context& c, int ik, const char* who);
int gamma_davidson_run(Context& c, int ik, int nbnd, double tol, int maxiter, double2* psio, double* eig_out,
                       int* iters_out, double* resnorm_out);
void gamma_release(Context& c);
// Nonlocal term of the Gamma form in real-basis coordinates (x: nb bands of nr = 2 nh reals, float
// or double; scaled = false: half-sphere coefficients, converted on load).  The float64 form writes
// out[b][r] = sum_p betar[p][r] (D' <betar|x>)[b][p]; the mixed form leaves float partial sums
// [*nsplit][nb][nr] (to be added in float64) in the mixed workspace and points *part at them.
int gamma_nonlocal_fp64(Context& c, const Problem& p, const void* x, bool x32, int nb, bool scaled, double* out);
int gamma_prepare_tc(Context& c, Problem& p);
// The projection half in float64 (w = D' <betar|x>, real form; w = D <beta|psi>, complex form),
// left in the workspace, and add_vuspsi from such a w on the tensor cores (mixed contexts).
int gamma_w_fp64(Context& c, const Problem& p, const void* x, bool x32, int nb, bool scaled, double** w);
// The same w with calbec as a double-float GEMM on the float32 pipes (needs d_betar_df)
int gamma_w_df(Context& c, const Problem& p, const void* x, bool x32, int nb, bool scaled, double** w);
int gamma_prepare_df(Context& c, Problem& p);
int nonlocal_w_fp64(Context& c, const Problem& p, const double2* psi, int nbnd, double2** w);
int gamma_add_tc(Context& c, const Problem& p, const double* w, int nb, const float** part, int* nsplit);
int nonlocal_add_tc(Context& c, const Problem& p, const double2* w, double2* hpsi, int nbnd);
int gamma_nonlocal_mixed(Context& c, const Problem& p, const void* x, bool x32, int nb, bool scaled,
                         const float** part, int* nsplit);
void scf_release(Context& c);
void fock_release(Context& c);

// ---- complex64 subspace products on the bf16 tensor cores (subspace_gemm.cu) ----
// Three-term bf16 split of a complex64 matrix's columns, kept valid up to `valid` columns.
struct SplitBasis {
  __nv_bfloat16* terms[3] = {nullptr, nullptr, nullptr};
  size_t cap = 0;
  int valid = 0;
  const float2* base = nullptr;
  int lds = 0;
  int ensure(Context& c, const float2* src, int ld, int cols);
  void invalidate() { valid = 0; }
  void release();
};
struct SubspaceGemm {
  __nv_bfloat16* bt[3] = {nullptr, nullptr, nullptr};
  float* P = nullptr;
  size_t bcap = 0, pcap = 0;
  int grow(Context& c, size_t bterms, size_t pfloats);
  // C (m x n) = alpha A^H B + beta C with A (k x m, lda) split through `split`; C64 (if not null)
  // is written instead of C32
  int ah_b(Context& c, cublasHandle_t h, int m, int n, int k, SplitBasis& split, const float2* A, int lda,
           const float2* B, int ldb, float alpha, float beta, float2* C32, double2* C64, int ldc);
  // C (M x n) = alpha A B + beta C with A (M x k, lda) split through `split`
  int a_b(Context& c, cublasHandle_t h, int M, int n, int k, SplitBasis& split, const float2* A, int lda,
          const float2* B, int ldb, float alpha, float beta, float2* C, int ldc);
  void release();
};

// ---- reduced Hermitian eigenproblem (eigh.cu) ----
bool eigh_supported(const Context& c, int n);
// Library kernels; *fallback is set (and nothing is wrong) when the caller should use cuSOLVER.
int eigh_lowest(Context& c, const double2* a, int lda, int n, int nwant, double* w_out, double2* v_out,
                bool* fallback);
// The solver chosen by HPSI_OPT_EIGENSOLVER, with cuSOLVER zheevdx behind the library kernels.
int eigh_reduced(Context& c, const double2* a, int lda, int n, int nwant, double* w_out, double2* v_out);
void eigh_release(Context& c);
// Real symmetric form (the reduced problems of the Gamma-point Davidson): the library's kernels for
// n up to 1824 on 152 SMs; *fallback as above.  Vectors to v_out [nwant][n] (column-major, ld n).
bool eigh_supported_real(const Context& c, int n);
int eigh_lowest_real(Context& c, const double* a, int lda, int n, int nwant, double* w_out, double* v_out,
                     bool* fallback, bool vec32 = false, bool df = false);

}  // namespace hpsi

// The opaque handle of the C ABI.
struct hpsi_ctx {
  hpsi::Context c;
};
