/*
 * hpsi.h -- plane-wave H|psi> and block-Davidson eigensolver on one GB300 (sm_103a).
 *
 * C ABI of libhpsi.so.  The operator is the Kohn-Sham Hamiltonian at fixed potential in a
 * plane-wave basis (paper Sec. 3; KS equation of App. A.1), available as an operator that
 * returns H|psi> for any block of states (App. A.2, Eq. (diag), with S = I for
 * norm-conserving separable projectors):
 *
 *     (H psi)(G) = |k+G|^2/2 psi(G)                                   kinetic (diagonal)
 *                + N_r^-1 sum_j e^{-iG.r_j} V(r_j) sum_G' e^{+iG'.r_j} psi(G')   local, via 3-D FFTs
 *                + sum_pq beta_p(G) D_pq sum_G' conj(beta_q(G')) psi(G')         separable nonlocal
 *
 * Units: Hartree atomic units (energies in Ha, lengths in bohr, k and G in 1/bohr).
 *
 * Conventions shared by every entry point
 *   - cell[9]: rows a1, a2, a3 of the lattice, row-major.  b = 2 pi (A^-1)^T.
 *   - G-sphere of a k-point: {G = m1 b1 + m2 b2 + m3 b3 : |k+G|^2/2 <= ecut} (inclusive, float64),
 *     ordered lexicographically by the signed Miller indices (m1, m2, m3).  hpsi_gsphere()
 *     returns this list; every psi / beta array is indexed in this order.
 *   - FFT grid: r_j = sum_i (j_i / n_i) a_i; V(r) is given as V[j1][j2][j3] (C order, j3 fastest).
 *     The sphere must map one-to-one into the box: n_i >= 2 max|m_i| + 1 (else HPSI_EINVAL).
 *   - Complex data are interleaved (re, im) float64 pairs (C99 double complex layout).
 *   - Wavefunction blocks are band-major: psi[b][g], b < nbnd, g < npw(k), no padding.
 *   - Every call is thread-compatible, not thread-safe: one context per host thread.
 *   - Return value: HPSI_OK (0) or a negative status; nothing aborts and no exception crosses
 *     the ABI.  hpsi_last_error() gives a one-line message for the last failure on a context
 *     (or, for a NULL context, for the last failure of this thread before a context existed).
 */
#ifndef HPSI_H
#define HPSI_H

#include <stdint.h>

#if defined(__GNUC__)
#define HPSI_API __attribute__((visibility("default")))
#else
#define HPSI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hpsi_ctx hpsi_ctx; /* opaque, owned by the library */

enum hpsi_status {
  HPSI_OK = 0,
  HPSI_EINVAL = -1,     /* bad argument (size, pointer, box too small, index out of range) */
  HPSI_ENOMEM = -2,     /* device or host allocation failed */
  HPSI_ECUDA = -3,      /* a CUDA runtime / library call failed (message in hpsi_last_error) */
  HPSI_ENOTCONV = -4,   /* davidson_solve reached maxiter; outputs hold the last iterate */
  HPSI_ESINGULAR = -5,  /* the reduced overlap matrix could not be factorised */
  HPSI_ETIMEOUT = -6,   /* a bounded device-side wait gave up (device error word set) */
  HPSI_ENODEV = -7      /* no usable sm_103 device */
};

enum hpsi_option {
  HPSI_OPT_PRECOND_TAU = 1,
  HPSI_OPT_PRECOND_SHIFT = 2,
  HPSI_OPT_KERNEL_TIMING = 3, /* 1: bracket every launch of the library's kernels with CUDA events */
  HPSI_OPT_NL_TERMS = 4,      /* mixed path: bf16 terms per nonlocal operand, 3 (six products,
                                 default) or 2 (three products); re-splits the projectors */
  HPSI_OPT_LOCAL_PATH = 5,    /* 0 (default): register-codelet kernels where the box allows them;
                                 1: always the generic radix-2/3/4/5 kernels */
  HPSI_OPT_TC_KSPLIT = 6,     /* mixed path: at most this many 64-wide K steps accumulate in one
                                 tensor-memory accumulator of <beta|psi> before the partial sums
                                 are added in float64 (0, default: at most 16, fewer where the
                                 output tiles alone would not fill the GPU) */
  HPSI_OPT_FINAL_FP64 = 7,    /* mixed davidson_solve(_gamma): the final Rayleigh quotients after one
                                 more application of H to the Ritz vectors.  2 (default): with float64
                                 projections <beta|psi> and D, the local term at the working precision
                                 and add_vuspsi on the tensor cores with one K-step per float32
                                 partial (the projections' error enters the quotients at first
                                 order; ~5e-8 Ha on the 144^3 cell); 1: with the float64 H (~3e-9 Ha);
                                 0: with the mixed H (~2e-6 Ha) */
  HPSI_OPT_BASIS = 8,         /* davidson_solve: the reduced basis grows to this many times N
                                 vectors (2: the basic 2N form, 3 or 4) before a restart; 0
                                 (default): 3 in a mixed context, 4 in a float64 one */
  HPSI_OPT_AUTOTUNE = 9,      /* 1 (default): the first hpsi_apply of a problem with >= 4 bands at a
                                 precision times every shared-memory plan of the register-codelet
                                 kernels and three band-block sizes on its own bands and keeps the
                                 fastest (results do not depend on the choice); at HPSI_MIXED it
                                 also times caps of 4, 8 and 16 K-steps per float32 accumulation of
                                 the tensor-core calbec (unless HPSI_OPT_TC_KSPLIT is set; results
                                 differ at float32 rounding level).  That call synchronizes.
                                 0: fixed defaults */
  HPSI_OPT_EIGENSOLVER = 10,  /* reduced eigenproblems of davidson_solve and hpsi_eigh_lowest:
                                 1 (default): the library's own kernels (Householder reduction,
                                 Sturm multisection, inverse iteration, back-transformation) for
                                 n <= 1024, cuSOLVER zheevdx above that or if inverse iteration
                                 loses a vector; 0: cuSOLVER zheevdx always */
  HPSI_OPT_FP32_GEMM = 11,    /* mixed davidson_solve (complex form): complex64 subspace GEMMs (projections, reduced
                                 matrices, Ritz vectors) 0 (default): float32 on the CUDA cores;
                                 1: float32 emulated by cuBLAS with bf16 tensor-core products
                                 (three bf16 terms per operand, nine products); 2: the Gauss
                                 three-product complex form (CGEMM3M); 3: the library's split:
                                 three bf16 terms per operand, six products accumulated in float32
                                 by bf16 tensor-core GEMMs, on the interleaved storage read as real
                                 matrices (the basis splits are cached across the iteration); 4: the
                                 inner products (projections onto the basis, H_sub columns, overlaps)
                                 on the library's tcgen05 kernel, three bf16 terms per float32
                                 operand (exact), six products, float32 accumulation per K-split and
                                 float64 sums over splits; the outer products stay CGEMM */
  HPSI_OPT_LOCKING = 12,      /* mixed davidson_solve: hard locking of converged Ritz pairs.  0: none
                                 (converged bands get no correction but stay in the Rayleigh-Ritz
                                 problem); 1: the lowest run of converged bands is frozen, taken out
                                 of the reduced basis, and later corrections are orthogonalised
                                 against it; 2: every converged band is frozen that way.  A lock
                                 restarts the reduced basis from the remaining Ritz vectors. */
  HPSI_OPT_LOCK_BATCH = 13,   /* a lock is taken once at least this fraction (0..1, default 0: one
                                 band) of the active bands is lockable */
  HPSI_OPT_LOCK_BASIS = 14,   /* after the first lock the reduced basis grows to at most this many
                                 times the active band count (>= 2, default 4) before a restart,
                                 and never past HPSI_OPT_BASIS times N */
  HPSI_OPT_THICK_RESTART = 15, /* davidson_solve: 0: a restart (or a lock) keeps the wanted (active)
                                 Ritz vectors; 1 (default): it keeps the lowest non-locked Ritz
                                 vectors up to half the basis limit (at least the active ones).  A
                                 mixed solve whose largest residual has not fallen by 10% in 8
                                 iterations continues with plain restarts, and if it stalls again
                                 restarts with H applied afresh to the kept vectors */
  HPSI_OPT_RITZ_SPLIT = 16,   /* mixed davidson_solve: 1: the Ritz-vector and restart products
                                 (inner dimension = basis size) run as float32 GEMMs over at most 8
                                 chunks of the inner dimension whose results are added in float64;
                                 0 (default): one float32 GEMM */
  HPSI_OPT_REORTH_TEST = 17,  /* davidson_solve: 1: the unit corrections are projected out of the
                                 basis once, and a second time only if a column kept less than half
                                 its squared norm; 0 (default): always twice */
  HPSI_OPT_CG_TMIN = 18,      /* cg_solve: the preconditioner is P^2 = 1 / max(|k+G|^2 / 2, value),
                                 value > 0 in Ha (default 1) */
  HPSI_OPT_SCF_NMIX = 19,     /* hpsi_scf: past (input density, residual) pairs the mixing combines
                                 (1..16, default 8) */
  HPSI_OPT_SCF_BETA = 20,     /* hpsi_scf: step along the optimal residual (0 < value <= 1, default 0.5) */
  HPSI_OPT_SCF_DAVIDSON_TOL = 21, /* hpsi_scf: residual tolerance of the Davidson solve of each
                                 iteration (default 1e-9) */
  HPSI_OPT_GAMMA_GEMM = 22,   /* mixed davidson_solve_gamma: 1 (default): the float32 subspace GEMMs
                                 run as cuBLAS's float32 emulation with bf16 tensor-core products
                                 (float32-accurate); 0: float32 on the CUDA cores */
  HPSI_OPT_EIGH_DF = 23,      /* real symmetric reduced problems.  1 (default): in the mixed
                                 davidson_solve_gamma the Householder reduction works in double-float
                                 arithmetic (pairs of float32, ~1e-13 relative, on the float32 pipes)
                                 and the eigenvectors' Gram, Newton-Schulz and back-transformation
                                 GEMMs in float32, since they rotate a float32 basis; float64 elsewhere.
                                 0: float64 throughout.  2: the double-float reduction also in
                                 hpsi_eigh_lowest_sym and the float64 davidson_solve_gamma (float64
                                 eigenvector GEMMs) */
  HPSI_OPT_PERSISTENT = 24,   /* hpsi_apply_batch: 1: one persistent cooperative launch per box edge
                                 (<= 32 items each) when every item has the register-codelet
                                 kernels; 0 (default): one launch per kernel class and box edge.
                                 The results are identical; the separate launches, replayed from a
                                 CUDA graph, are faster since each kernel runs at its own occupancy */
  HPSI_OPT_BATCH_NL = 25      /* hpsi_apply_batch in a mixed context: the nonlocal term.  0 (default):
                                 in float64 on the CUDA cores, one launch per kernel class over all
                                 items, when every item has at most 64 projectors, else 1.  1: the
                                 tensor-core form per item.  2: always the float64 batched form */
};

/* Kernel classes reported by hpsi_kernel_stats. */
enum hpsi_kernel {
  HPSI_K_INV_ZY = 0,   /* scatter + inverse z and y transforms per m1-plane */
  HPSI_K_XVX_Y = 1,    /* inverse x, x V(r), forward x, forward y per z-plane */
  HPSI_K_FWD_Z = 2,    /* forward z, gather, kinetic term per m1-plane */
  HPSI_K_CALBEC = 3,   /* <beta|psi> (split-K partial sums) */
  HPSI_K_DSCALE = 4,   /* reduction of the partials and D <beta|psi> */
  HPSI_K_ADDVUS = 5,   /* hpsi += beta (D <beta|psi>) */
  HPSI_K_SPLIT = 6,    /* mixed path: bf16 operand splitting */
  HPSI_K_DAVIDSON = 7, /* Davidson residual / preconditioner / helper kernels */
  HPSI_K_EIGH = 8,     /* reduced eigenproblem: multisection, inverse iteration,
                          back-transformation helpers */
  HPSI_K_TRIDIAG = 9,  /* reduced eigenproblem: the Householder reduction to tridiagonal form */
  HPSI_K_GAMMA = 10,   /* Gamma-point form: packing two real bands into one complex band, unpacking */
  HPSI_K_SCF = 11,     /* self-consistency loop: density, full-box transforms, Hartree, LDA, mixing,
                          potential update */
  HPSI_K_FOCK = 12,    /* exchange operator: sphere <-> box maps, codensities, full-box transforms,
                          Coulomb kernel, sums over occupied bands */
  HPSI_K_BATCH = 13,   /* hpsi_apply_batch: the persistent launch over every item (local term and,
                          in float64, the nonlocal term) */
  HPSI_K_COUNT = 14,
  HPSI_K_AT_FP64 = 16  /* added to a class in hpsi_kernel_stats: only the launches made while H (or,
                          for the nonlocal classes, its nonlocal term) was applied in float64: all
                          of them in a float64 context; in a mixed context the final float64
                          application of davidson_solve and the float64 nonlocal term of a batch
                          (HPSI_OPT_BATCH_NL) */
};

enum hpsi_precision {
  HPSI_FP64 = 0,  /* every step in float64 / complex128 */
  HPSI_MIXED = 1  /* FFTs and x V(r) in float32, nonlocal contractions as split-bf16
                     tensor-core GEMMs with float32 accumulation (three bf16 terms per operand,
                     six products, by default; a batch of items with few projectors takes the
                     float64 form, HPSI_OPT_BATCH_NL); kinetic term in float64.  davidson_solve keeps
                     its reduced basis in complex64 and does the small eigensolves, the residual
                     norms and the final Rayleigh quotients in float64 */
};

/*
 * hpsi_gsphere -- the plane-wave basis at one k-point (paper Sec. 3, PW basis |k+G> of App. A.2.1).
 *   cell[9]      in   lattice rows (bohr)
 *   ecut         in   kinetic cutoff (Ha), > 0
 *   k_cart[3]    in   k in Cartesian coordinates (1/bohr)
 *   npw_out      out  number of plane waves
 *   miller_out   out  nullable; if not NULL, receives [npw][3] int32 Miller indices in the
 *                     documented order, provided capacity >= npw (else HPSI_EINVAL, npw_out set)
 *   capacity     in   rows available in miller_out
 * Host only; touches no GPU.
 */
HPSI_API int hpsi_gsphere(const double cell[9], double ecut, const double k_cart[3], int* npw_out,
                 int32_t* miller_out, int capacity);

/*
 * hpsi_setup -- build the operator for one cell and nk k-points (paper Sec. 3 and App. A.1-A.2).
 *   out          out  new context (NULL on failure)
 *   cell, ecut        as in hpsi_gsphere
 *   nk           in   number of k-points, >= 1
 *   kpts         in   host [nk][3] Cartesian k-points (1/bohr)
 *   fft[3]       in   FFT box n1, n2, n3 (each 2*3*5-smooth, 8 <= n <= 256)
 *   vloc_r       in   host float64 [n1][n2][n3], the local potential V(r_j) (Ha), real
 *   nproj        in   number of projectors P >= 0 (same for every k)
 *   beta         in   host complex128: for k = 0..nk-1 in order, a block [P][npw(k)] of beta_p(k+G);
 *                     ignored (may be NULL) when P = 0
 *   dmat         in   host complex128 [P][P], Hermitian (only its nonzeros are used)
 *   precision    in   HPSI_FP64 or HPSI_MIXED
 *   cuda_stream  in   cudaStream_t (NULL = legacy default stream) on which all work is queued
 * The library copies every input to device memory it owns; the caller may free them on return.
 * Problem index ik of later calls is the k-point index.
 */
HPSI_API int hpsi_setup(hpsi_ctx** out, const double cell[9], double ecut, int nk, const double* kpts,
               const int fft[3], const double* vloc_r, int nproj, const double* beta,
               const double* dmat, int precision, void* cuda_stream);

/*
 * hpsi_setup_cells -- one context over ncell independent cells, each at Gamma (k = 0), each with
 * its own box, potential and projectors (the many-small-cells batch).  Arguments are arrays
 * over cells: cells [ncell][9], ecut [ncell], fft [ncell][3], vloc_r[c] host [n1][n2][n3],
 * nproj [ncell], beta[c] host complex128 [P_c][npw_c] (NULL if P_c = 0), dmat[c] host
 * complex128 [P_c][P_c].  Problem index ik of later calls is the cell index.
 */
HPSI_API int hpsi_setup_cells(hpsi_ctx** out, int ncell, const double* cells, const double* ecut,
                     const int* fft, const double* const* vloc_r, const int* nproj,
                     const double* const* beta, const double* const* dmat, int precision,
                     void* cuda_stream);

/* Number of problems (k-points or cells) in a context, and npw / nproj of problem ik
 * (negative status on a bad index). */
HPSI_API int hpsi_nprob(const hpsi_ctx* ctx);
HPSI_API int hpsi_npw(const hpsi_ctx* ctx, int ik);
HPSI_API int hpsi_nproj(const hpsi_ctx* ctx, int ik);

/*
 * hpsi_apply -- hpsi_out = H psi_in for a block of nbnd bands of problem ik
 * (the operator of App. A.2, Eq. (diag); terms as in the file header).
 *   psi_in       in   complex128 [nbnd][npw(ik)]
 *   hpsi_out     out  complex128 [nbnd][npw(ik)]; must not overlap psi_in
 *   nbnd         in   >= 0 (0 is a no-op)
 * Either both pointers are device memory (then the call is asynchronous on the context's
 * stream) or both are host memory (then the library stages them through device buffers it
 * owns and returns after the result has been copied back).  Mixed host/device pairs are
 * HPSI_EINVAL.  The library allocates its device workspace on first use and keeps it.
 */
HPSI_API int hpsi_apply(hpsi_ctx* ctx, int ik, const void* psi_in, void* hpsi_out, int nbnd);

/*
 * hpsi_apply_noalloc -- the same H psi as hpsi_apply, for callers that cannot let the library
 * allocate device memory during the call.  The paper has no counterpart; this exists for
 * integration: some callers have all device memory reserved up front by another allocator (a
 * framework's caching pool, a fixed per-process budget), and some cannot accept the device-wide
 * synchronisation that cudaMalloc / cudaFree imply in the middle of an asynchronous pipeline.
 *   psi_in, hpsi_out  device memory only (host pointers are HPSI_EINVAL: staging them would need
 *                     buffers), complex128 [nbnd][npw(ik)], not overlapping
 * Every intermediate lives in one fixed 64 MiB array compiled into the library; every GPU that
 * loads libhpsi.so holds those 64 MiB until the process exits.  Bands are processed in chunks that
 * fit it; if a single band's intermediates exceed 64 MiB the call returns HPSI_EINVAL (use
 * hpsi_apply).  The nonlocal term uses the float64 kernels at both precisions.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  Every call shares the one
 * array and leaves its contents behind (each call writes every byte it later reads, so nothing
 * has to start cleared): calls whose work can overlap on the GPU -- two streams, or two contexts
 * -- race on it and must be serialised by the caller.  Asynchronous on the context's stream.
 */
HPSI_API int hpsi_apply_noalloc(hpsi_ctx* ctx, int ik, const void* psi_in, void* hpsi_out, int nbnd);

/*
 * hpsi_apply_gamma -- H psi for real orbitals at k = 0, half the components stored (paper Sec. 4,
 * the Gamma-point trick of PWscf).
 *   psi_in, hpsi_out  complex128 [nbnd][nh], nh = (npw(ik) + 1) / 2: the coefficients c(G) of the
 *                     half sphere S+, which is the last nh entries of the sphere's order: G = 0
 *                     first (its coefficient must be real; an imaginary part is ignored), then
 *                     every G whose first nonzero Miller index is positive.  c(-G) = conj(c(G))
 *                     is implied.  Device (asynchronous) or host (synchronous) memory, as in
 *                     hpsi_apply; must not overlap.
 * Two bands share one complex transform pair and one pass of the nonlocal contractions: with
 * f = psi_a + i psi_b, F = H f, (H psi_a)(G) = (F(G) + conj F(-G)) / 2 and
 * (H psi_b)(G) = (F(G) - conj F(-G)) / (2i).  Valid when H maps real functions to real ones; the
 * library checks at setup that problem ik is at k = 0, that its sphere is symmetric, and that each
 * projector has beta_p(-G) = u_p conj(beta_p(G)) with |u_p| = 1 and conj(u_p) u_q conj(D_pq) = D_pq
 * (true for real-Y_lm projectors with any per-projector phase and real diagonal D); otherwise
 * HPSI_EINVAL with the reason in hpsi_last_error.  Counts nbnd band-applications.
 */
HPSI_API int hpsi_apply_gamma(hpsi_ctx* ctx, int ik, const void* psi_in, void* hpsi_out, int nbnd);

/*
 * davidson_solve_gamma -- davidson_solve for real orbitals at k = 0 (paper Sec. 4 with the block
 * Davidson of App. A.2.1).
 *   psi_inout    in/out complex128 [nbnd][nh] half-sphere coefficients (as hpsi_apply_gamma),
 *                     device or host; initial guess in, orthonormal real eigenvectors out
 *   other arguments as in davidson_solve (nbnd times the basis factor must not exceed npw)
 * The real orbital with half coefficients c is the real vector x = (c(0), 0) at G = 0 and
 * sqrt2 (Re c(G), Im c(G)) elsewhere; inner products are x_a . x_b and H is real symmetric, so the
 * subspace products are real GEMMs (float64 in a float64 context; float32 in a mixed one, by default
 * emulated on the bf16 tensor cores, HPSI_OPT_GAMMA_GEMM) and the
 * reduced problems real symmetric (float64, the library's real eigensolver as in
 * hpsi_eigh_lowest_sym, cuSOLVER dsyevdx behind it).  Residual norms and Cholesky
 * factors are float64; the preconditioner uses <G|H|G> for both coordinates of each G.  In a mixed
 * context the returned eigenvalues are float64 Rayleigh quotients after one float64 application of
 * H (HPSI_OPT_FINAL_FP64).  HPSI_OPT_BASIS, _THICK_RESTART, _PRECOND_TAU, _PRECOND_SHIFT and
 * _GAMMA_GEMM apply; locking and HPSI_OPT_FP32_GEMM do not.  Synchronous; HPSI_ENOTCONV if maxiter is reached.
 */
HPSI_API int davidson_solve_gamma(hpsi_ctx* ctx, int ik, int nbnd, double tol, int maxiter, void* psi_inout,
                                  double* eig_out, int* iters_out, double* resnorm_out);

/*
 * hpsi_apply_batch -- H psi for several problems (k-points or cells) in one launch sequence:
 * for i < nitem: hpsi_out[i] = H(prob[i]) psi_in[i] with nbnd[i] bands.  Device pointers only.
 * Items whose cubic box has register-codelet kernels share one launch of each local-potential
 * kernel per box edge (blockIdx.z runs over the items), and the nonlocal term follows: one launch
 * per kernel class over all items in float64, which a mixed context also takes when every item has
 * at most 64 projectors (HPSI_OPT_BATCH_NL), else the tensor-core form per item.  With
 * HPSI_OPT_PERSISTENT = 1, and every item on those kernels, each box edge (<= 32 items) is instead
 * one persistent cooperative launch whose CTAs take tiles from per-phase work lists: the
 * z-scatter/inverse transforms, the plane transforms with x V, the forward transforms and gather,
 * and in a float64 context the nonlocal calbec, D and add_vuspsi of its items, with a bounded grid
 * barrier between the phases (an expired wait sets the error word that hpsi_sync reports as
 * HPSI_ETIMEOUT).  Both forms give the same results bit for bit.
 * The first call with a given argument list runs eagerly and captures the same sequence in a CUDA
 * graph; later calls with identical arguments (same problems, band counts and pointers) replay
 * the graph with one launch.  Items are independent; outputs must not overlap inputs or each other.
 * (Pools of k-points and task groups of bands in the paper's Table 1 are prior art for this
 * batching; here the items simply share the launches of one GPU.)
 */
HPSI_API int hpsi_apply_batch(hpsi_ctx* ctx, int nitem, const int* prob, const int* nbnd,
                     const void* const* psi_in, void* const* hpsi_out);

/*
 * davidson_solve -- lowest nbnd eigenpairs of H for problem ik by block Davidson with the
 * diagonal preconditioner (App. A.2.1).
 *   nbnd         in   number of bands N (1 <= N, and N * basis factor <= npw; factor 3 in a mixed
 *                     context, 4 in a float64 one, HPSI_OPT_BASIS)
 *   tol          in   convergence when max_i ||H psi_i - eps_i psi_i||_2 <= tol
 *   maxiter      in   iteration limit (>= 1)
 *   psi_inout    in/out complex128 [N][npw(ik)], device or host: initial guess in (need not be
 *                     orthonormal, must be linearly independent), orthonormal eigenvectors out
 *   eig_out      out  host float64 [N], ascending eigenvalues (Ha)
 *   iters_out    out  nullable; iterations taken
 *   resnorm_out  out  nullable; host float64 [N], final residual norms
 * Steps: orthonormalise psi (Cholesky); repeat { residuals g_i = (H - eps_i) psi_i and their
 * norms; corrections D g_i with <k+G|D|k+G> = 1/(<k+G|H|k+G> - eps_i) (denominator kept at
 * |.| >= 0.1 Ha); orthogonalise them against the reduced basis and add them; H_jk, S_jk of the
 * reduced basis; solve (H - eps S) c = 0 in float64; psi_i <- sum_j c_j phi_j; when the basis
 * would exceed its limit restart from the lowest Ritz vectors (up to half the limit,
 * HPSI_OPT_THICK_RESTART; hard locking with HPSI_OPT_LOCKING) }.  At HPSI_MIXED the
 * basis is complex64 and the returned eigenvalues are float64 Rayleigh quotients (see
 * HPSI_OPT_FINAL_FP64); the returned residual norms are those of the returned vectors.
 * Synchronous: returns when done.
 * HPSI_ENOTCONV if maxiter is reached (outputs then hold the last iterate).
 */
HPSI_API int davidson_solve(hpsi_ctx* ctx, int ik, int nbnd, double tol, int maxiter, void* psi_inout,
                   double* eig_out, int* iters_out, double* resnorm_out);

/*
 * cg_solve -- lowest nbnd eigenpairs of H for problem ik by the band-by-band preconditioned
 * conjugate-gradient minimisation of App. A.2.2.
 *   nbnd, psi_inout, eig_out, resnorm_out  as in davidson_solve, except that eig_out and the rows
 *                     of psi_inout come in the order the bands were found (ascending when every
 *                     band reached its minimum)
 *   tol          in   a band stops when ||H psi - eps psi||_2 <= tol
 *   maxiter      in   step limit per band (>= 1)
 *   iters_out    out  nullable; CG steps over all bands (one application of H to one band each)
 * Band i starts from row i of psi_inout, orthogonalised to the bands j < i and normalised; each
 * step takes lambda = <psi|P^2 H|psi> / <psi|P^2|psi>, the gradient P^2 (H - lambda) psi
 * orthogonalised to the bands j < i, a Polak-Ribiere direction orthogonalised to psi, and the
 * exact minimum of <psi|H|psi> on psi cos t + n sin t.  P^2 = 1 / max(|k+G|^2/2, t_min) is the
 * kinetic-only preconditioner (t_min: HPSI_OPT_CG_TMIN, 1 Ha).  Float64 vectors; H is applied at
 * the context's precision.  Synchronous.  HPSI_ENOTCONV if a band reaches maxiter (outputs then
 * hold the last iterate).
 */
HPSI_API int cg_solve(hpsi_ctx* ctx, int ik, int nbnd, double tol, int maxiter, void* psi_inout,
                      double* eig_out, int* iters_out, double* resnorm_out);

/*
 * hpsi_scf -- the self-consistency loop of App. A.1 around davidson_solve, for problem ik of a
 * float64 context (its local potential as given at setup is V_ext).
 *   nocc         in   occupied bands (two electrons each), >= 1
 *   nbnd         in   bands solved each iteration, nocc <= nbnd (extra bands help the eigensolver)
 *   tol          in   stop when the scf norm ||rho_out - rho_in||^2 < tol (Ha), with
 *                     ||a||^2 = 4 pi Omega sum_{G != 0} |a(G)|^2 / G^2 (twice the Hartree energy of a)
 *   maxiter      in   iteration limit
 *   psi_inout    in/out complex128 [nbnd][npw(ik)], device or host: starting orbitals, then the
 *                     orbitals of the last iteration
 *   rho_inout    in/out host float64 [n1][n2][n3]: the starting density rho_in (electrons per bohr^3
 *                     on the grid), then the converged input density
 *   eig_out      out  host float64 [nbnd]: eigenvalues of the last iteration's H
 *   energies_out out  host float64 [2]: E = sum_i f_i eps_i - int rho_out V_Hxc[rho_in] + E_Hxc[rho_out]
 *                     and the Harris-Weinert-Foulkes E' with rho_in in place of rho_out (no ion-ion
 *                     term); they agree at self-consistency
 *   iters_out    out  nullable: iterations taken
 *   norm2_out    out  nullable host float64 [maxiter]: ||rho_out - rho_in||^2 of each iteration
 * Each iteration: V = V_ext + V_H[rho_in] + V_xc[rho_in] (V_H(G) = 4 pi rho(G) / G^2, V_H(0) = 0;
 * LDA: Slater exchange and the Perdew-Zunger parametrisation of the Ceperley-Alder correlation) is
 * written into the context; davidson_solve (tolerance HPSI_OPT_SCF_DAVIDSON_TOL) from the previous
 * orbitals; rho_out = sum_{i < nocc} 2 |psi_i(r)|^2 / Omega; the next rho_in is the combination of
 * the last HPSI_OPT_SCF_NMIX inputs whose combined residual has the smallest scf norm, plus
 * HPSI_OPT_SCF_BETA times that residual (the Anderson form).  On return the context's potential is
 * V[rho_in] of the last iteration, so hpsi_apply applies the self-consistent H.  The density is that
 * of problem ik alone.  Synchronous.  HPSI_ENOTCONV if maxiter is reached (outputs hold the last
 * iterate).
 */
HPSI_API int hpsi_scf(hpsi_ctx* ctx, int ik, int nocc, int nbnd, double tol, int maxiter, void* psi_inout,
                      double* rho_inout, double* eig_out, double* energies_out, int* iters_out, double* norm2_out);

/*
 * hpsi_fock_apply -- the Fock exchange operator at the Gamma point (paper App. A.5) applied to a
 * block of bands, for closed shells: with phi = psi / Omega^(1/2),
 *     (V_x psi_b)(r) = - sum_j psi_j(r) v_bj(r),  v_bj = Coulomb potential of conj(psi_j) psi_b / Omega,
 *     v(G) = 4 pi n(G) / G^2 (G != 0),  v(0) = 4 pi n(0) x_div,
 *     x_div = Omega / (2 pi)^3 * 2 pi^(3/2) / alpha^(1/2) - sum_{G != 0 in the FFT box} e^{-alpha G^2} / G^2
 * (the Gygi-Baldereschi treatment of the q -> 0 divergence with the auxiliary function
 * e^{-alpha G^2} / G^2 for the single q point; the 0/0 term the paper estimates from a coarser q grid
 * is left out).  Codensities are formed on the full FFT box.
 *   ik           in   a problem at k = 0 (else HPSI_EINVAL)
 *   nocc, occ    in   device complex128 [nocc][npw]: the occupied orbitals (two electrons each)
 *   psi_in       in   device complex128 [nbnd][npw]
 *   vx_out       out  device complex128 [nbnd][npw]: (V_x psi)(G) on the sphere; must not overlap
 *                     occ or psi_in
 *   alpha        in   exponent of the auxiliary function (bohr^2), > 0 (1 is the usual choice)
 *   ex_out       out  nullable host double: Re sum_b <psi_b|V_x psi_b>; with psi_in = occ this is the
 *                     exchange energy E_x = - sum_ij (ij|ji) of the occupied set (synchronizes)
 * Asynchronous on the context's stream when ex_out is NULL.  Float64 throughout.
 */
HPSI_API int hpsi_fock_apply(hpsi_ctx* ctx, int ik, int nocc, const void* occ, const void* psi_in, void* vx_out,
                             int nbnd, double alpha, double* ex_out);

/*
 * hpsi_eigh_lowest -- the lowest nwant eigenpairs of a dense Hermitian matrix: the reduced
 * problem sum_k (H_jk - eps S_jk) c_k = 0 that the Rayleigh-Ritz step of block Davidson solves
 * over its orthonormal reduced basis (App. A.2.1; S_jk is then the identity).  davidson_solve
 * calls the same solver; this entry point exposes it on its own.
 *   n            in   order of the matrix, >= 1
 *   a            in   device complex128, column-major with leading dimension lda >= n; only the
 *                     upper triangle (row <= column) is read and the imaginary parts of the
 *                     diagonal are ignored; not modified
 *   nwant        in   1 <= nwant <= n
 *   w_out        out  device double[nwant], eigenvalues ascending
 *   v_out        out  device complex128 [nwant][n] (column-major n x nwant, leading dim n):
 *                     orthonormal eigenvectors, each determined up to a phase (and, within a
 *                     degenerate eigenvalue, up to a unitary mixing)
 * Float64 throughout.  With HPSI_OPT_EIGENSOLVER = 1 (default) and n <= 1024: Householder
 * reduction to a real tridiagonal T (one cooperative launch with bounded grid-barrier waits),
 * Sturm multisection for the eigenvalues of T, inverse iteration with Gram-Schmidt inside
 * clusters of close eigenvalues and Cholesky QR for the eigenvectors, back-transformation;
 * otherwise cuSOLVER zheevdx.  Synchronizes the context's stream.  HPSI_EINVAL on bad sizes or
 * pointers, HPSI_ETIMEOUT if a barrier wait ran out, HPSI_ECUDA / HPSI_ENOMEM on CUDA failures,
 * HPSI_ESINGULAR if zheevdx fails.
 */
HPSI_API int hpsi_eigh_lowest(hpsi_ctx* ctx, int n, const void* a, int lda, int nwant, void* w_out, void* v_out);

/*
 * hpsi_eigh_lowest_sym -- hpsi_eigh_lowest for a real symmetric matrix: the reduced problem of the
 * Rayleigh-Ritz step when the reduced basis is real (davidson_solve_gamma, paper Sec. 4 with
 * App. A.2.1).
 *   a            in   device float64, column-major, leading dimension lda >= n; upper triangle read
 *   w_out        out  device double[nwant], ascending
 *   v_out        out  device float64 [nwant][n] (column-major n x nwant, leading dim n): orthonormal
 *                     eigenvectors, each up to a sign (and a rotation within a degenerate eigenvalue)
 * Float64.  Real Householder reduction to tridiagonal form (one cooperative launch, a quarter of the
 * float64 work of the complex one), Sturm multisection, inverse iteration, real compact-WY
 * back-transformation.  n up to 1824 on 152 SMs (the rows must fit their shared memory), otherwise
 * HPSI_EINVAL; also HPSI_EINVAL if inverse iteration loses a vector (davidson_solve_gamma then uses
 * cuSOLVER dsyevdx).  Synchronizes the context's stream.
 */
HPSI_API int hpsi_eigh_lowest_sym(hpsi_ctx* ctx, int n, const void* a, int lda, int nwant, void* w_out, void* v_out);

/*
 * hpsi_set_option -- tune the Davidson solver of a context (App. A.2.1, the diagonal form of D).
 *   HPSI_OPT_PRECOND_TAU    value > 0 (Ha): denominators <k+G|H|k+G> - eps of D are kept at
 *                           |.| >= value (default 0.1).
 *   HPSI_OPT_PRECOND_SHIFT  0 (default): eps = eps_i, the band's own Ritz value (D approximates
 *                           (H - eps_i S)^-1);  1: one eps for every band, the highest Ritz value
 *                           of the block (the estimate of the highest occupied eigenvalue).
 * HPSI_EINVAL for an unknown option or a bad value.  Host only.
 */
HPSI_API int hpsi_set_option(hpsi_ctx* ctx, int option, double value);

/*
 * hpsi_kernel_stats -- launches of the library's own kernels on ctx since the last reset, and
 * (with HPSI_OPT_KERNEL_TIMING on) their summed device time in ms from the bracketing events.
 *   kernel       in   an hpsi_kernel value (plus HPSI_K_AT_FP64 for its float64-precision launches
 *                     only), -1 for all classes together (total_ms then 0),
 *                     -2 for the number of H|psi> band-applications performed (in launches), or
 *                     -3 for the reduced eigenproblems solved by the library's own eigensolver
 *                     (in launches) and how many of them it handed to cuSOLVER (in total_ms), or
 *                     -4 for the tridiagonal reductions run by the library (in launches) and
 *                     their algorithmic float64 work, sum of 16 n^3 / 3 real flops (in total_ms)
 *   launches     out  nullable; number of launches
 *   total_ms     out  nullable; summed event time (synchronizes the context's stream)
 *   reset        in   non-zero: clear the counters after reading
 * cuBLAS / cuSOLVER kernels of the Davidson subspace algebra are not counted.
 */
HPSI_API int hpsi_kernel_stats(hpsi_ctx* ctx, int kernel, long long* launches, double* total_ms, int reset);

/*
 * hpsi_sync -- wait for all work queued on the context's stream, then report a device-side
 * failure: HPSI_ETIMEOUT if a bounded wait inside a library kernel expired since the last
 * check (the affected outputs are invalid; the error word is cleared).  Synchronous host-pointer
 * calls and davidson_solve make the same check themselves.
 */
HPSI_API int hpsi_sync(hpsi_ctx* ctx);

/*
 * hpsi_selftest_timeout -- exercise the device failure path: queue on the context's stream a
 * one-thread kernel that waits, with a limit of about 2e6 cycles (~1 ms), on a shared-memory
 * barrier nothing ever arrives at, the same bounded wait the tensor-core kernels use; on expiry it
 * raises the context's error word and returns.  The next hpsi_sync reports HPSI_ETIMEOUT (and
 * clears the word).  Nothing faults or hangs; the context stays usable.
 */
HPSI_API int hpsi_selftest_timeout(hpsi_ctx* ctx);

/* One-line message for the last failure on ctx (NULL ctx: this thread's last setup failure). */
HPSI_API const char* hpsi_last_error(const hpsi_ctx* ctx);

/* Free every device and host resource of ctx (NULL is a no-op).  Synchronizes its stream. */
HPSI_API void hpsi_destroy(hpsi_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HPSI_H */
