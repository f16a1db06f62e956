"""CPU oracle for the plane-wave H|psi> hot path and its block-Davidson solver (FP64).

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the package ``paper_0906_2569_gb300``
and its CUDA library) imports, links or calls this package.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / ``--impl reference`` legs use
it.  It shares no code with the CUDA path; both take their inputs from ``workloads``.

What it computes is the plain definition of each step, in float64 / complex128:

* ``gsphere``   -- the plane-wave basis {G : |k+G|^2/2 <= E_cut}, the kinetic diagonal
                   (paper Sec. 3; PW notation of App. A.2.1).
* ``hamiltonian`` -- H|psi> = T psi + [V psi] + sum_pq |beta_p> D_pq <beta_q|psi>, both via a
                   full-box FFT (scipy) and as a dense matrix H_GG' built element by element
                   with a direct (non-FFT) DFT of V (KS equation of App. A.1; the operator form
                   of Eq. (diag) in App. A.2; separable projectors of Sec. 3).
* ``davidson``  -- the per-step quantities of the block Davidson method of App. A.2.1:
                   residuals g_i = (H - eps_i S) psi_i with S = I, the diagonal correction
                   D g_i, and the Rayleigh-Ritz solve of the reduced problem.
* ``cg``        -- the band-by-band preconditioned conjugate-gradient eigensolver of App. A.2.2
                   (constrained minimisation per band, kinetic-only P^2, Polak-Ribiere
                   directions, exact line minimum on the unit circle).
* ``scf``       -- the self-consistency loop of App. A.1 around H|psi>: density, Hartree and LDA
                   potentials, the scf norm, the mixing of past densities, and the standard and
                   Harris-Weinert-Foulkes energies.
* ``gamma``     -- the Gamma-point real-wavefunction form (Sec. 4): half-sphere storage, the real
                   basis in which H is real symmetric, two real bands per complex FFT.
* ``fock``      -- Fock exchange at Gamma (App. A.5): codensity potentials by FFT, the
                   Gygi-Baldereschi treatment of the G = 0 divergence, V_x psi and E_x.
* ``eigen``     -- reference eigenvalues: dense LAPACK ``eigh`` of H_GG' (small cells) and
                   scipy LOBPCG on the FFT H|psi> (large cells).

Pins (tests/test_oracle_pins.py) tie these to facts fixed outside the oracle: closed forms
(free electrons, the analytic Fourier transform of the Gaussian wells, the secular equation
of a rank-one projector), brute-force O(N^2) sums with Cartesian G.r, invariants
(Hermiticity, rigid translation, k -> k + b, k -> -k) and library routines on tiny inputs.
The absolute eigenvalues of the synthetic cells have no printed value in the paper: they
are pinned only through those properties and the agreement of two independent routes.
"""
from . import gsphere, hamiltonian, davidson, eigen, cg, scf, gamma, fock  # noqa: F401
