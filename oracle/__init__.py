"""FP64 CPU oracle for grid hopping (Monnoyer et al., "Grid Hopping:
Accelerating Direct Estimation Algorithms for Multistatic FMCW Radar").

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it. The product path (the CUDA
library and its Python binding) never imports, calls or links anything here,
and this package never imports the product.

Everything is plain NumPy in float64 / complex128, written from the paper's
equations in the paper's order, with library primitives (matrix products,
``lstsq``) as single steps and no blocking or fusion:

* ``model``   - sensing functions and atoms (Eq. 1, Sec. II), measurement
                synthesis (Eq. general-model);
* ``maps``    - zero-padded 2D DFT range-Doppler maps (Sec. III, Sec. IV);
* ``hopping`` - polar interpolation coefficients, coordinate table, hopping
                score and argmax (Eq. 5, Sec. IV);
* ``direct``  - exact direct decision function, brute force and factored
                (Eqs. 3-4, Sec. III);
* ``bomp``    - block OMP detect-and-deflate loop (Sec. VI, future work).

Readings of the paper where it is silent or ambiguous are stated in each
function's docstring. Parity status: every function is pinned by a test in
``tests/test_oracle_*.py`` against closed forms, invariants, brute force or a
library routine; none is "parity unpinned".
"""
from . import model, maps, hopping, direct, bomp  # noqa: F401
