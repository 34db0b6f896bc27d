"""Plain FP64 CPU oracle for rapid Kriging prediction.

TEST INFRASTRUCTURE ONLY. Nothing in the product path (the package
``paper_2605_29284_gb300`` and its CUDA library) imports, links or runs this
package; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it.

The oracle restates, slowly and directly, what the paper "Rapid Approximation
Prediction for Kriging" (Li, Fasshauer, Nychka) computes:

* ``matern``  -- the Matern covariance of Eq. (Matern1), Section 3.
* ``kriging`` -- exact Kriging, Eqs. (2)-(5), Section 2.
* ``rapid``   -- the rapid approximation, Eqs. (6)-(9) and steps 1-7 of the
                 algorithm in Section 2.2, evaluated by direct summation of
                 Eq. (9) (a naive dense BTTB product, no FFT), plus a literal
                 step-7 version that uses a library FFT as a primitive.
* ``philox``  -- Philox4x64-10 (Salmon et al., SC'11) and the Box-Muller map,
                 the counter-based noise of conditional simulation.
* ``cs``      -- conditional simulation, Section 1 and Section 5.2.
* ``grad``    -- the adjoint of the implemented approximate map (the paper has
                 no gradient; the derivation is stated in ``grad``).

Every function is FP64. Pins that tie it to the paper and to mathematics
rather than to itself live in ``tests/test_oracle_*.py``.
"""
