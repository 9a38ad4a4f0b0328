"""Plain, slow, FP64 CPU oracle for the binary-lens evolutionary fitter of Rajpaul (2012).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package: only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.
It shares no code with the CUDA library (``paper_1208_4830_gb300``) and imports nothing
from it; both sides receive their inputs from ``paper_1208_4830_gb300.synth``, which holds
none of the method's arithmetic.

Modules
-------
``sblm``    forward model of Section 2.2: trajectory (Eq. sourcePos), lens equation
            (Eq. lensing), quintic (Eq. lensingPoly, coefficients derived here),
            roots, spurious-root rejection, image magnification and the chi^2 of Section 4.1.
``philox``  Philox4x64-10 counter-based generator (Salmon et al. 2011), the random source of
            every stochastic EA operator on both sides.
``ea``      the evolutionary algorithm of Appendix A, operator by operator, in the
            paper's order, plus a reference driver.
``cnn``     the learned proposal network (not in the paper: this project's seeding of the
            initial population), forward and backward by hand in FP64.
``polish``  the amoeba (downhill simplex) fine-tuning of the fittest solution, Section 4.1.
``proposal`` the proposal's data path: training curves, binning, initial weights, AdamW,
            and seed rows encoded as genes.

Parity status (see each module's header): the forward model and the EA operators are
pinned by tests under ``tests/`` that do not re-type the oracle's formulas; whole EA runs
are judged statistically because rank ties flip under floating-point reordering.
"""
