"""Oracle: a plain, slow, FP64 CPU trust-region-reflective curve fit.

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may call it.  It shares no code with the CUDA path (no kernels, headers,
constants or helpers); the two meet only on the seeded inputs drawn by
``paper_2208_12187_gb300.synth``.

Contents
  models.py  h(x; p) and the analytic partials dh/dp for the four models,
             vectorised NumPy FP64 (Section 2, Eqs. residual and jacobian);
             any callable (X, p) -> (h, dh/dp) stands for a user-defined model.
  reduce.py  the per-evaluation quantities written from their definitions:
             r, J, cost f = r^T r / 2 (Eq. msqe), g = J^T r (Eq. gradient),
             B = J^T J (Eq. hessian, Gauss-Newton term), with 1/sigma row
             weighting (Appendix C, Eqs. easy_jac, easy_res).
  trf.py     the fit itself: Algorithm 1 (outer loop), Algorithm 2 (LM
             parameter), Algorithm 3 (acceptance and radius), Eq. accuracy
             (ratio), Appendix B (thin SVD of the scaled Jacobian), the
             Coleman-Li reflective treatment of bounds that Section 2 cites
             without detail, termination tests and pcov.

Parity status per function (what pins it; see tests/test_oracle_*.py):
  models.*             central differences; exact linear-model Jacobian;
                       a callable equal to a built-in gives the built-in's fit
  reduce.evaluate      finite-difference gradient of the cost; Gauss-Newton
                       Hessian equals the true Hessian on noise-free data;
                       sum of split pieces equals the whole
  trf.lm_parameter     More-Sorensen conditions (Eqs. lm, pbound); bisection
                       root of phi; np.linalg.solve of (B + a I) p = -g
  trf.tr_radius_update Algorithm 3 tables
  trf.curve_fit        linear model == normal equations; noise-free data ==
                       truth; zero projected gradient; monotone cost; bounds
                       feasibility; infinite bounds == unbounded; SciPy's
                       least_squares optimum (a library run, same minimiser)
  trf.select_bounded_step  parity unpinned by the paper (Section 2 names the
                       Coleman-Li method but does not state it); pinned only by
                       the invariants above and KKT conditions at active bounds.
"""
from . import models, reduce, trf  # noqa: F401
