"""FP64 CPU oracle for the real-space Kohn-Sham LOBPCG path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference legs may import this package.  The
product path (the CUDA library and its Python binding) never imports, calls or
links it, and this package imports nothing from the product path: the two share
no code.  The only common module is ``workloads`` (seeded raw inputs).

Everything here is plain NumPy/SciPy in float64 / complex128, written to be
checked against the paper by eye:

* ``grid``        -- grid, G-vectors, Gaussian local potential, KB projectors
* ``hamiltonian`` -- H psi = T psi + V psi + sum |beta> E <beta|psi>  (SCF tasks
                     (1) and (4) of the paper: FFT Laplacian, nonlocal operator)
* ``linalg``      -- the Cholesky + two-TRSM reduction of Eq. 1 and the
                     subspace eigensolve (SCF task (3))
* ``lobpcg``      -- Knyazev's LOBPCG with the Rayleigh-Ritz of Eq. 1 (SCF
                     tasks (2)-(3)) and the Teter-Payne-Allan preconditioner
* ``precond``     -- the learned preconditioner: a residual-form periodic 3D
                     convolutional network on TPA, its gradient, Adam, and the
                     projected correction targets by MINRES
* ``tddft``       -- real-time propagation by the Taylor series of exp(-i H dt)
* ``gga``         -- PBE exchange-correlation (the paper's functional), FFT gradients
* ``gamma``       -- the real-arithmetic Gamma-point LOBPCG (real orbitals, real
                     transforms, real Gram matrices, real-symmetric Eq. 1)
* ``scf``         -- density, FFT Hartree, LDA (Slater + Perdew-Zunger 1981),
                     occupations (aufbau / Fermi-Dirac), Anderson mixing, and
                     one SCF step (the "Others" component of Fig. 1)

Every function is pinned by tests in ``tests/test_oracle_*.py`` against
closed forms, invariants, library routines and brute force; see each module's
header for the pins and for the functions that are parity-unpinned.
"""
