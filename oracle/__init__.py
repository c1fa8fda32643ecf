"""Plain FP64 CPU oracle of the EnKF-MC analysis step (test infrastructure).

This package is the checker, not the product.  Only the tests, the smoke
check of `__graft_entry__` and the CPU-baseline leg of `bench.py` may import
it.  It shares no code with the CUDA library: its geometry, regressions,
assembly and solves are written out here from the paper (Nino, Sandu, Deng,
"A Parallel Implementation of the Ensemble Kalman Filter Based on Modified
Cholesky Decomposition", 2016):

  Section 2.1, Eq. 1-3   modified Cholesky: regress each component on its
                         predecessors; T holds -beta, D the residual variances
  Section 2.3, Eq. 5     ensemble anomalies U = Xb - mean
  Section 2.3, Eq. 8-9   B^-1 ~ T^T D^-1 T, B ~ T^-1 D T^-T
  Section 2.3, Eq. 10-11 primal analysis increment
  Section 2.3, Eq. 12-13 dual analysis increment
  Section 3, Eq. 14, Algorithms 2-3  sub-domain analysis with an r-wide
                         boundary that is discarded after the local solve
  Algorithm 1, Eq. 18    filter cycling with a synthetic forecast operator
                         (advection) and the analysis RMSE (cycling.py)

Floating point is float64 throughout.  Library routines (matrix products,
Cholesky factorisation, triangular and sparse solves) serve as single steps;
there is no blocking, fusion or reordering beyond what the equations state.
"""
from .enkfmc import (Grid, Subdomain, anomalies, perturbed_observations, regress, estimate,
                     estimate_rows, subdomains, local_estimate, local_system, local_analysis,
                     analysis, assimilate, b_hat_dense, gain_form_analysis, dual_form_analysis,
                     dual_increment, local_dual_analysis, t_pattern_csr, rel_err)
from .cycling import forecast_shift, ensemble_sqerr, rmse_eq18, filter_cycles

__all__ = ["Grid", "Subdomain", "anomalies", "perturbed_observations", "regress", "estimate",
           "estimate_rows", "subdomains", "local_estimate", "local_system", "local_analysis",
           "analysis", "assimilate", "b_hat_dense", "gain_form_analysis", "dual_form_analysis",
           "dual_increment", "local_dual_analysis", "t_pattern_csr", "rel_err", "forecast_shift", "ensemble_sqerr", "rmse_eq18",
           "filter_cycles"]
