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

Parity unpinned in part (no value from the paper fixes which of two
consistent readings is taken; stability chose, and the implementation of the
reading is pinned):
  * the exterior current at an interface (`dg.external_fd_current`,
    `fd.fill_ghosts` for J~): the neighbour's current transferred like its
    state, not the current of the transferred state.  Pinned at DG-FD faces
    by the exactness of the mixed right-hand side with a linear current, and
    at faces between wedges by the eta-independence of a force-free state
    (tests/test_oracle_curved.py, tests/test_oracle_schemes.py).
FD ghosts across a neighbour's face are, by default (prm["ghost_interp"], set
by Problem, the reading the CUDA path implements), the neighbour's data
interpolated to this element's grid extension; the neighbour's own cells
(ghost_interp off) agree inside a wedge and on boxes and are inconsistent
between cubed-sphere wedges (tests/test_oracle_curved.py).
The rollback bookkeeping of a substep redone on FD (`stepper`) is pinned on
fields linear in x: a step with switches after substeps A, B and C equals the
step without them.  The star boundary state (`physics.bc_star`) is pinned by a
static dipole that stays put; the shells of the black-hole tests may live in
spherical Kerr-Schild coordinates (`geometry.ShellMesh(spin=a)`, App. B),
pinned by the spheroid relation, the paper's time step on the vacuum Wald grid
and King's horizon flux (`surface`); the exact-Wald errors of Table II are
reproduced with the outflow face inside the horizon.
"""
