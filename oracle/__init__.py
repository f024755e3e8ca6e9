"""CPU oracle for the complex-coordinate FMM (test infrastructure only).

This package is the plain, slow, obviously-correct CPU statement of what the
GPU path computes. It shares no code with the CUDA library and imports
nothing from it. Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it; the
product path never calls it.

Modules
-------
direct   : the direct O(NM) sums (Eqs. lap_2d_pot, helm_2d_pot, lap_3d_pot,
           the 3D Helmholtz sum of Sec. 5.3, and their double-layer forms,
           Sec. 2.1), in float64 / complex128. Parity pinned (tests/test_oracle_direct.py).
tree     : tree on the real parts, level restriction, complexified centres,
           Lists 1-4 (Sec. 6.1-6.2) and expansion orders (Sec. 6.3).
           Parity pinned (tests/test_oracle_tree.py).
fmm2d    : the 2D Laplace and 2D Helmholtz complex-coordinate FMMs (Sec. 4,
           Sec. 6.4). Parity pinned (tests/test_oracle_fmm2d.py).
"""
