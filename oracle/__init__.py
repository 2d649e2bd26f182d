"""Plain, slow FP64 CPU oracle for the axisymmetric drift-diffusion-Poisson solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it, and it shares no code with the CUDA
path: it is an independent restatement of the paper's equations in numpy /
scipy so that every GPU result can be checked against it.

Modules (each function cites the passage it follows):

* ``grid``            - the (r, z) node set and finite-volume geometry (Sec. 2,
                        eqs. 12-13 fix the control volumes).
* ``bernoulli``       - F(x), G(x) of the Scharfetter-Gummel flux (after eq. 11).
* ``discretization``  - face fluxes (eqs. 8-11), the backward-Euler residual
                        (eq. 7) and the Poisson rows (eqs. 12-13), and the
                        Newton Jacobian with 3x3 blocks (eq. 14).
* ``multigrid``       - the V-cycle used to solve eq. 14 (Sec. 2 names the
                        multigrid method only; the components are the readings
                        listed in this project's design notes).
* ``solver``          - Newton-Raphson time step, the Delta-t ramp with
                        rejection, and the coarse-to-fine steady continuation
                        ("multilevel prolongation", Sec. 2 and the abstract).

Parity pins live in ``tests/test_oracle_*.py``.  Functions without a pin say
"parity unpinned" in their docstring.
"""
from . import bernoulli, grid, discretization, multigrid, solver  # noqa: F401
