"""FP64 CPU oracle for the RT-TDDFT propagation of Jakowski et al. (arXiv:2410.09189).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.  The
CUDA library never calls it and shares no code with it; the only common module is
``paper_2410_09189_gb300.inputs``, which produces seeded inputs and holds none of the
method's arithmetic.

Plain, slow, obviously-correct NumPy/SciPy in float64, written from the paper:

* ``fd``          -- central finite-difference Laplacian (Section 2.1, Eq. 2).
* ``hamiltonian`` -- grid, local Gaussian-erf wells, Kleinman-Bylander projectors, H applied
                     to orbitals (Eq. 1 with the grid quadrature of Eq. 4).
* ``poisson``     -- Hartree potential of the discrete 12th-order operator (Section 2.1).
* ``lda``         -- Slater exchange + Perdew-Zunger 1981 correlation.
* ``groundstate`` -- SCF ground state that supplies the active-space orbitals
                     (Algorithm 1's ground state).
* ``tddft``       -- Algorithm 1: commutator expansion (Eqs. 19, 32-33), Hamiltonian
                     self-consistency, linear extrapolation, kick (Eq. 34), dipole.
* ``gridprop``    -- the occupied orbitals propagated on the grid, the complete-grid-basis
                     limit of Algorithm 1 (Section 2.2).
* ``spectrum``    -- absorption spectrum (dipole strength function) from the kicked dipole
                     series of the three kick directions (Section 4).
* ``surrogate``   -- learned correction to the linear-extrapolation seed of the SCF loop
                     (Algorithm 1's extrapolation): conv3d network, its gradient, Adam.

Parity status of each function is stated in its module header.
"""
