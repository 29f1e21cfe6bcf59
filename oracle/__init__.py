"""FP64 CPU oracle for the mapped Legendre / Fourier pseudo-spectral hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
Python binding) may import, call or link this package; only the tests, the smoke
check and the CPU-baseline leg of the benchmark use it.  It shares no code with the
GPU path: every quantity here (nodes, weights, basis, operators, transforms,
solves, integrators) is computed afresh in plain numpy/scipy FP64.

What it follows (paper: "MLegS: a modern mapped Legendre spectral method solver
for unbounded domains", Lee & Wang):

* grid.py        -- algebraic map Eq. (1), Gauss-Legendre nodes (Sec. 3.1)
* basis.py       -- normalised associated Legendre functions, Eq. (7) (Sec. 3.1)
* transform.py   -- truncated expansion Eq. (2) and its quadrature inverse
* operators.py   -- horizontal Laplacian Eqs. (4)-(5), r d/dr, dissipation Eq. (11)
* integrate.py   -- FE-BE and AB-CN Eq. (12) with Richardson start (Sec. 3.3),
                    Fisher-KPP reaction Eq. (17)
* vortex.py      -- toroidal-poloidal velocity/vorticity Eq. (8), projection Eq. (9),
                    nonlinear term of Eq. (19)
* diagnostics.py -- weighted L2 norm, circulation and second moment Eq. (16)
* filter.py      -- adaptive modal filter applied between steps (Sec. 3.3)
* surrogate.py   -- FP64 reference of the learned surrogate's network, its
                    backward pass and Adam (not in the paper; gradient reference)

Pins (the tests under tests/test_oracle_*.py): library Gauss nodes, discrete
orthonormality, library associated Legendre values, two independent Laplacian
constructions and a hand-derived closed form, exact round trips, azimuthal purity,
the paper's printed representation errors (Sec. 5.1), every digit of Table 2
(Oseen), the Fisher-KPP linearised errors (Sec. 5.2), closed-form diffusion, and
vortex-projection invariants.  Functions with no pin say "parity unpinned".
"""

from .grid import Grid, gauss_legendre, map_r  # noqa: F401
from .basis import pbar_table, ln_norm  # noqa: F401
from .transform import (forward, backward, to_flat, from_flat,  # noqa: F401
                        spec_zeros, spec_norm, spec_rel_err)
from .operators import (del2h_closed, del2h_quadrature, rdr_matrix,  # noqa: F401
                        linear_operator)
from .integrate import Stepper, fkpp_nonlinear  # noqa: F401
from .diagnostics import weighted_l2, l2w, circulation, second_moment  # noqa: F401
from .vortex import VortexOps, vortex_nonlinear  # noqa: F401
from . import surrogate  # noqa: F401
from . import filter as modal_filter  # noqa: F401
