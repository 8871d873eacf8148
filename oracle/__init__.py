"""CPU FP64 oracle for the superblock H*psi + Lanczos path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  It shares no code with the CUDA library and never imports it; its
only common dependency with the GPU side is the seeded input container in
``workloads/``.

Plain, slow, obviously correct NumPy/SciPy code in float64, following the
paper (G. Alvarez, "The Density Matrix Renormalization Group for Strongly
Correlated Electron Systems: A Generic Implementation"):

* ``models``    site operators and lattice Hamiltonians (Sec. 4.1, Sec. 1)
* ``ed``        exact diagonalisation of a whole lattice (brute force)
* ``superblock`` explicit Kronecker superblock (Sec. 3.3) and the
                sector-blocked product x += H y (Sec. 3.3, tasks i-iii)
* ``lanczos``   Lanczos ground state with full reorthogonalisation
* ``grad``      transpose product, coefficient gradients, Hellmann-Feynman
* ``dmrg``      infinite (Sec. 3.1, Fig. infiniteloop) and finite algorithm

Parity pins: every module is pinned in ``tests/test_oracle_*.py`` against
closed forms, the paper's printed energies, brute force on tiny inputs or
invariants; see each function's docstring.
"""
