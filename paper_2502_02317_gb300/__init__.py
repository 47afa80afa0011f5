"""GB300-native boundary-MPS PEPS contraction and branch-and-bound search for
clustered Ising / Potts models (arXiv:2502.02317, SpinGlassPEPS.jl).

The work runs in ``libspg`` (CUDA, sm_103a) behind the C ABI of
``include/spg.h``; this package is its ctypes binding.
"""
import os as _os

# spg_solve_batch overlaps up to 32 worker streams, which needs as many
# hardware work queues (CUDA's default is 8); the variable is read when the
# process creates its CUDA context, so import this package before the first
# CUDA call for it to apply.  A value set by the user is kept.
_os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

from ._binding import (SPG_ECUDA, SPG_EINEXACT, SPG_EINVAL, SPG_ENOMEM, SPG_ENUMERIC, SPG_ETIMEOUT,
                       SPG_EUNSUPPORTED, SPG_FP64, SPG_KING, SPG_MIXED, SPG_SQUARE, SPG_TUNE_FORCE, SPG_TUNE_OFF,
                       SPG_TUNE_ON, SPG_WS_FEATURES, Context, Mlp, Problem, Result,
                       SpgError, lib, params, spg_boundary_export, spg_debug_marginals, spg_lattice_site_map,
                       spg_check_bounded_wait, spg_inject_alloc_failure, spg_log_partition,
                       spg_peak_probe, spg_problem_ising, spg_problem_potts, spg_profile,
                       spg_profile_report,
                       spg_problem_update_ising, spg_set_warm_start, spg_solve, spg_solve_batch, spg_solve_group,
                       spg_solve_lattice8, spg_sweep_trace, spg_tc_product, spg_truncate, spg_autotune_clear,
                       spg_autotune_report, spg_autotune_set, spg_potts_hamiltonian, Hamiltonian,
                       spg_diversity,
                       spg_truncate_static, spg_warm_features)

__all__ = ["Context", "Problem", "Result", "SpgError", "lib", "params", "spg_problem_ising",
           "spg_problem_potts", "spg_solve", "spg_solve_batch", "spg_solve_group", "spg_debug_marginals", "spg_log_partition",
           "spg_profile", "spg_profile_report", "spg_tc_product", "spg_truncate", "spg_lattice_site_map",
           "spg_truncate_static", "spg_warm_features", "spg_boundary_export", "Mlp", "spg_set_warm_start",
           "spg_sweep_trace", "SPG_WS_FEATURES", "spg_peak_probe", "spg_check_bounded_wait",
           "spg_inject_alloc_failure", "spg_solve_lattice8", "spg_problem_update_ising",
           "spg_autotune_set", "spg_autotune_clear", "spg_autotune_report", "SPG_TUNE_OFF", "SPG_TUNE_ON",
           "SPG_TUNE_FORCE", "spg_potts_hamiltonian", "Hamiltonian", "spg_diversity",
           "SPG_FP64", "SPG_MIXED", "SPG_SQUARE", "SPG_KING", "SPG_EINVAL", "SPG_EINEXACT", "SPG_ENOMEM",
           "SPG_ECUDA", "SPG_ETIMEOUT", "SPG_ENUMERIC", "SPG_EUNSUPPORTED"]
