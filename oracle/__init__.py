"""CPU oracle for the D2Q37 thermal lattice-Boltzmann step (arXiv:1703.04594).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_1703_04594_gb300``) never imports, calls or links anything here and fails
loudly when its CUDA library is missing.

The oracle is a plain, slow, float64 transcription of the method:

* ``oracle.d2q37``  - the velocity set, the lattice weights and scale factor (solved
  here from the isotropy conditions) and the Hermite-expanded equilibrium, written as
  explicit tensor contractions.
* ``oracle.lbm``    - moments (Sec. 3, eq. ``macro``), BGK collision with the gravity
  shift (eq. ``lbequation``), pull-scheme propagate (eq. ``master2``), thermal-wall
  boundary condition, a full step, initialisation and the kinetic-energy observable.

It shares no code, table or constant with the CUDA path; only the seeded input
generator (``paper_1703_04594_gb300.inputs``, which holds none of the method's
arithmetic) feeds both.

Parity status per function (what pins it; see ``tests/test_oracle_*.py``):

* weights / scale ``c``: isotropy residuals, positivity, normalisation.
* ``equilibrium``: all moments up to order 4 equal the continuous Maxwellian's closed
  form; the Hermite tensor form agrees with the scalar expansion at random points.
* ``collide``: mass/momentum/energy conservation (g = 0), exact momentum kick
  rho*g and unchanged temperature (g != 0), equilibrium fixed point.
* ``propagate``: permutation + round trip under reversed velocities, brute-force
  index check on a 4x8 lattice.
* ``bc``: wall-equilibrium fixed point at rest, linearity in f, and a hand-computed
  ghost value on a tiny lattice.
* RT initial state inputs: hydrostatic balance checked against the continuous
  closed form on unperturbed columns.
"""
