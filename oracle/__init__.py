"""FP64 CPU oracle of the Monte Carlo KBC lattice Boltzmann method.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this package; the product
package never does.  The stepper lives in ``lbm_oracle.c`` (plain C, FP64 and
an FP64-complex twin for complex-step derivatives); the ensemble statistics
live in ``stats.py`` (NumPy).  Neither shares code with the CUDA library.
"""
from .build import build_oracle, load_oracle  # noqa: F401
from .stepper import (  # noqa: F401
    lattice, units, equilibrium, collide, shear_part, init_ensemble, step, run, moments, energy, hrel,
    complex_step_grad, rtgv_fields, leray_project, init_ensemble_leray, exact_gamma,
)
