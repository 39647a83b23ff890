"""FP64 CPU oracle for the Multi-Frequency WaveHoltz (MFWH) method (arXiv 2507.23613).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
statement of what the GPU path computes.  Only the test suite, the smoke check
in ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product library never imports, links
or calls anything here, and this package imports nothing from the product.

Modules
-------
filters  -- set-up arithmetic: time step, adjusted frequencies (eq. omegaImplicit),
            period counts (eq. TbarDef), trapezoid weights (eq. DefNI), filter
            kernel (eq. newFilterKernel), traditional parameters
            (eq. origParamAdjust), least-squares parameters (Algorithm 2),
            filter weights (eq. pDefQ) and the filter matrix B (eq. filterA).
wave     -- the MFWH map Pi (Algorithm 1 body, explicit scheme eq. WaveScheme),
            fixed-point iteration, GMRES on A = I - S (eq. krylovSystem),
            Helmholtz residual (eq. errorAndResid), sparse direct Helmholtz
            solve and the closed-form Dirichlet spectrum used by the pins.

Every function is FP64 numpy; library primitives (lstsq, solve, spsolve) are
used as single steps.  Pins that tie this code to the paper live in
``tests/test_oracle_*.py``.
"""
