"""GB300 (sm_103a) Parareal for the two-asset Black-Scholes equation.

The compute path is the CUDA library libbsparareal.so (include/bsparareal.h); this package
is its thin Python binding.  Importing a function that needs the library loads it and fails
loudly if it cannot be built or loaded.
"""
from ._lib import (BASKET, CALL1, CASH_OR_NOTHING, COARSE_NUM, COARSE_PINO, EXCHANGE, EXPORTS,
                   OPT_COARSE_VARIANT, OPT_FINE_SWEEPS, OPT_JACOBI_TARGET, OPT_JACOBI_TARGET_COLD,
                   OPT_EXTRAP_LATE, OPT_EXTRAP_START, OPT_JACOBI_TARGET_EXTRAP,
                   OPT_JACOBI_TARGET_EXTRAP_LATE, OPT_KRYLOV_MAXIT, OPT_PIPELINE, OPT_KRYLOV_TOL, OPT_FINE_KRYLOV_TOL, OPT_FINE_TILE, OPT_PHASE_TIMING,
                   PARAREAL_USER_U0, START_COLD, START_EXTRAP, START_EXTRAP_LATE, START_WARM, BSError,
                   Grid, Pino, Server, bs_coarse_variant, bs_device_allocations, bs_coarse_variant_info, bs_payoff3, fine_propagate3, coarse_propagate3, parareal_solve3, bs_fine_steps_for, bs_fine_sweeps, bs_grid_stats, bs_payoff,
                   bs_phase_stats, bs_set_option, coarse_propagate, coarse_propagate_batched, fine_propagate_batched,
                   last_error, load, parareal_solve, parareal_solve_noalloc, parareal_sweep_range, pino_physics_loss,
                   to_params)

__all__ = ["BASKET", "CALL1", "CASH_OR_NOTHING", "COARSE_NUM", "COARSE_PINO", "EXCHANGE",
           "EXPORTS", "OPT_COARSE_VARIANT", "OPT_FINE_SWEEPS", "OPT_JACOBI_TARGET",
           "OPT_JACOBI_TARGET_COLD", "OPT_EXTRAP_LATE", "OPT_EXTRAP_START", "OPT_JACOBI_TARGET_EXTRAP",
           "OPT_JACOBI_TARGET_EXTRAP_LATE", "OPT_PIPELINE", "OPT_KRYLOV_MAXIT", "OPT_KRYLOV_TOL", "OPT_FINE_KRYLOV_TOL", "OPT_FINE_TILE", "OPT_PHASE_TIMING",
           "PARAREAL_USER_U0", "START_COLD", "START_EXTRAP", "START_EXTRAP_LATE", "START_WARM", "BSError", "Grid", "Pino", "Server", "bs_coarse_variant", "bs_device_allocations", "bs_coarse_variant_info", "bs_payoff3", "fine_propagate3", "coarse_propagate3", "parareal_solve3", "bs_fine_steps_for", "bs_fine_sweeps",
           "bs_grid_stats", "bs_payoff", "bs_phase_stats", "bs_set_option", "coarse_propagate", "coarse_propagate_batched",
           "fine_propagate_batched", "last_error", "load", "parareal_solve",
           "parareal_solve_noalloc", "parareal_sweep_range", "pino_physics_loss", "to_params"]
