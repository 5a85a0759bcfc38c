"""FP64 reference oracle for the graph-based shadow-QMD hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
CPU restatement of what the method computes, written from the paper
(arxiv 2606.03140, "SEDACS: A Scalable Framework for Complex Chemistry
Simulations") and its supporting information.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The CUDA path never imports, links or
calls anything in here, and nothing in here imports the CUDA path: the two
share only the seeded input generators of ``paper_2606_03140_gb300.inputs``.

Modules
-------
sk       Slater-Koster sp blocks, their derivatives, H0 / S assembly
ewald    periodic Gaussian-gamma Coulomb matrix, potential and gradients (Ewald)
graph    distance + density threshold graph, recursive coordinate bisection, halos
density  subgraph solve (S^-1/2, Fermi operator), global mu, collection,
         Mulliken charges, shadow energy and forces
cjacobi  the plain-C parts: subgraph eigensolves by cyclic Jacobi rotations
         (csrc/jacobi.c; density's default route) and the bisection for mu on
         the collected count (csrc/mu.c), compiled with gcc
dynamics SCC with linear mixing, XL-BOMD integrator, low-rank Krylov kernel
gnn      message-passing preconditioner network, forward and backward

Parity status of each function is stated in its docstring ("pinned by ..."
or "parity unpinned").
"""

BOHR_A = 0.529177210903          # 1 bohr in Angstrom (CODATA 2018)
AU_TIME_FS = 0.02418884326585747  # 1 atomic time unit in fs
AMU_ME = 1822.888486209           # 1 amu in electron masses
KB_HA = 3.166811563e-6            # Boltzmann constant, Hartree / K
