"""Plain FP64 CPU oracle for the fluctuating non-ideal-fluid lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (no kernels, headers, constant tables or helpers).

The oracle follows Gross & Varnik, "Simulation of static critical phenomena in
non-ideal fluids with the Lattice Boltzmann method" (arXiv:1202.4748):

* ``philox``       -- Philox4x32-10 counter-based generator (Salmon et al., SC'11)
                      and Box-Muller normals; the paper only asks for Gaussian
                      variates (Sec. III A, text around Eq. 67).
* ``lattice``      -- D2Q9 velocity set, weights and moment basis (Sec. III A,
                      Eqs. 65-66, 68); D3Q19 set and an orthogonal basis
                      (literature variant, not in the paper).
* ``lbm``          -- one time step: moments (Eq. 62), modified equilibrium
                      (Eqs. 63-65), moment-space relaxation and noise (Eqs. 61,
                      66-68), periodic streaming; Guo-forced variant.
* ``observables``  -- block order parameter, susceptibility, specific heat
                      (Sec. II B, Eqs. 46-50) and the structure factor (Eq. 80).

Everything is float64.  Parity status of each function is stated in its
docstring; the pins live in ``tests/test_oracle_*.py``.  Items fixed by this
implementation's own conventions (velocity ordering, Philox counter layout,
gradient stencil, per-mode noise reading, initial condition) are
"parity unpinned" by the paper: GPU and oracle agree by construction there,
and the statistical / closed-form pins check that the choices reproduce the
paper's physics.
"""

from . import philox, lattice, lbm, observables  # noqa: F401
