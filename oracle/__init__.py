"""FP64 CPU oracle for the QUAPI tensor-propagator path -- TEST INFRASTRUCTURE ONLY.

This package is the slow, plain reference that the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference arm of ``bench.py`` may import it; the product path never does.  It
shares no code, header, table generator or constant with the CUDA library and
never imports the ``paper_1205_6872_gb300`` package.

What it computes (all FP64, hbar = k_B = 1):

* ``eta``        -- the eta coefficients of the discretised influence
  functional, as double integrals of the bath response function alpha(t)
  (Sec. II, Eq. bathResponseFunction and Eqs. etaKK'generalTrotter ..
  etaNkgeneralStrang), reduced to one frequency integral per box pair and
  evaluated by adaptive Gauss-Kronrod quadrature (QUADPACK via scipy).
* ``system``     -- the bare system propagator e^{-i H dt} and the
  forward/backward pair propagator K(x', x) of the path-integral expression
  for <s_N^+|rho(t)|s_N^-> (Sec. II).
* ``recurrence`` -- the tensor-propagator recurrence (Sec. I, Makri-Makarov
  scheme; memory length Delta k_max, Sec. II) written plainly: growth of the
  augmented tensor A for k < Delta k_max, then multiply-by-T and sum over the
  oldest path index, and the rho readout at the requested steps
  (allPoints / justFinalPoint, Sec. IV).  The inner loops are in
  ``quapi_oracle.c`` (plain C, OpenMP over output elements).
* ``bruteforce`` -- the truncated path sum itself, by explicit enumeration of
  every forward/backward path (tiny N only).

Pins (tests marked ``not gpu``): closed-form eta for the Ohmic bath at zero and
finite temperature, a direct 2-D integration of alpha(t) over the boxes, exact
unitary evolution for J = 0, the pure-dephasing (independent-boson) closed
form, brute force vs recurrence, and the trace / Hermiticity invariants.
Parity is unpinned beyond the oracle only for non-commuting H with J != 0 at
large memory length (no closed form exists and the paper prints no rho values).
"""

from .eta import Spectral, eta_boxes, eta_table, pack_eta, unpack_eta, strang_box  # noqa: F401
from .system import propagator_U, pair_propagator_K, coupling_d  # noqa: F401
from .recurrence import propagate, step_tables, readout_tables, OracleRun  # noqa: F401
from .bruteforce import rho_bruteforce  # noqa: F401
