"""Plain FP64 CPU oracle of the non-conforming IMEX-DG Euler solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` use it.  It shares no code with the CUDA
library; the two meet only through the seeded case descriptions of the
``workloads`` package.

The oracle is written for a reader checking it against the paper, not for
speed.  Element operators are dense Kronecker products (no sum
factorisation), hanging-face traces are evaluated by evaluating the coarse
cell's Lagrange polynomial at the fine face points, and the connectivity is
found by looking up neighbours in a dictionary of tree leaves.

Sections of the paper followed:

* Eq. (1) (Sec. 2): compressible Euler equations with gravity, ideal gas
  p = rho R T, g = 9.81, R = 287.
* Sec. 2, method paragraph: DG in space on non-conforming meshes without
  hanging nodes, IMEX-RK2 in time with energy and momentum coupled
  implicitly and continuity explicit; matrix-free operator action (Sec. 3.2).
* Sec. 3.1: orography profile, stratified background atmosphere (p formula
  read with the missing factor g restored), wall bottom boundary.
* Sec. 3.2: pressure fixed-point loop with GMRES for the non-symmetric
  linear system.

Every discretisation detail the paper defers to earlier work is a reading,
listed in the repository's design notes: GLL collocation, Rusanov flux,
the ARK2 tableau of Giraldo-Kelly-Constantinescu, the Helmholtz form of the
implicit stage and the subface treatment of 2:1 faces.

Parity status: every public function here is pinned by the ``-m "not gpu"``
tests in ``tests/test_oracle_*.py`` (closed forms, exactness, invariants,
brute force on tiny meshes).  One reading is only partly pinned: free-stream
preservation on *curved 3D hanging* faces is not exact for this
discretisation (collocated subface quadrature is not exact for curl-free
normals there); it is reported, not asserted.
"""
