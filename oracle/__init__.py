"""Plain FP64 CPU oracle for one IMEX Runge-Kutta step of the v-eta DNS method
for Taylor-Couette flow (Pirro & Quadrio, "Direct Numerical Simulation of
turbulent Taylor-Couette flow").

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and
the CPU-baseline leg of the benchmark may import it.  The CUDA product path
never imports, links or calls anything here, and this package imports nothing
from the product package.

What it computes, and where each piece comes from in the paper:

* grid.py       -- geometry, radial grid, Fourier mode sets (Sec. 2, Sec. 4,
                   Appendix: k^2 = alpha^2 + m^2/r^2).
* stencils.py   -- 5-point compact explicit radial stencils, coefficients from
                   polynomial matching (Sec. 2.1), built in exact rational
                   arithmetic and rounded once to FP64.
* fourier.py    -- Fourier expansion in theta and z, pseudo-spectral products
                   with the 3/2 rule (Appendix, "non-linear terms as written in
                   the original primitive-variables equations").
* operators.py  -- the radial rows of Eq. 6 (v), Eq. 7 (eta), the mean flow,
                   the velocity reconstruction from continuity, the boundary
                   conditions v = Dv = eta = 0 (Appendix).
* rk.py         -- the 3-substep IMEX Runge-Kutta step (Sec. 2.1, Sec. 3.1).
* diagnostics.py-- torque, Eq. 2 (reading fixed by Table 2), Re_tau (Sec. 5),
                   kinetic energy, and the energy budget the paper does not
                   print: viscous dissipation nu <2 S:S> and the power of the
                   wall shear (dE/dt = P_in - eps).
* linear.py     -- linearised operator of one Fourier mode about circular
                   Couette flow, used to pin the critical Reynolds numbers of
                   Sec. 3.

Every floating-point quantity is float64 (complex128 for spectral data).
Parity of a full step has no printed value in the paper; it is pinned
indirectly, piece by piece, by the tests in tests/test_oracle_*.py.
"""
from .grid import Case, radial_grid
from .stencils import Stencils, build_stencils
from .rk import SMR91, OracleSolver

__all__ = ["Case", "radial_grid", "Stencils", "build_stencils", "SMR91", "OracleSolver"]
