"""CPU oracle for the GRFFE DG-FD hybrid hot path (arXiv:2404.01531).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, fp64 (or complex128
for complex-step derivatives) restatement of the discretisation in the paper:
the 3+1 force-free system in conservative form (Sec. II), the nodal DG-SEM
operator with LGL collocation, mass lumping and the exponential filter
(Sec. III.A), IMEX-SSP3(4,3,3) time integration with the stiff current and
divergence-cleaning damping treated implicitly (Sec. III.B), the conservative
FD subcell scheme with WENO5-Z, Rusanov flux and the 4th-order derivative
corrector (Sec. III.C.2), the Persson-type troubled-cell indicator (Sec.
III.C.3) and the no-incoming-Poynting outer boundary (Sec. III.D).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The CUDA library never
links or calls anything here, and nothing here imports the CUDA package.

Every function cites the passage it follows.  Readings taken where the paper is
silent are marked ``[reading]`` in the docstrings.

Parity unpinned (no value from the paper or mathematics fixes them; they are
checked only by GPU-vs-oracle agreement, conservation and convergence):
  * at a face shared by a DG and an FD element, the exterior current
    (`dg.external_fd_current`, `fd.fill_ghosts` for J~: the projection of the
    current, a reading); the exterior state there (`dg.external_dg_state` with
    an FD neighbour, `fd.fill_ghosts` with a DG neighbour) is pinned by the
    exactness of the mixed DG/FD right-hand side on linear fields.
FD ghosts across a neighbour's face: copied from its cells (the default, the
reading the CUDA path implements) or, with prm["ghost_interp"], interpolated to
this element's grid extension; only the latter converges between cubed-sphere
wedges (tests/test_oracle_curved.py).
The rollback bookkeeping of a substep redone on FD (`stepper`) is pinned the
same way: on fields linear in x a step with switches after substeps A, B and C
equals the step without them.
"""
