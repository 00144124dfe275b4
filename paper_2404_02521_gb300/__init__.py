"""GB300 (sm_103a) Parareal for the two-asset Black-Scholes equation.

The compute path is the CUDA library libbsparareal.so (include/bsparareal.h); this package
is its thin Python binding.  Importing a function that needs the library loads it and fails
loudly if it cannot be built or loaded.
"""
from ._lib import (BASKET, CALL1, CASH_OR_NOTHING, COARSE_NUM, COARSE_PINO, EXCHANGE, EXPORTS,
                   BSError, Grid, Pino, bs_fine_sweeps, bs_payoff, coarse_propagate,
                   fine_propagate_batched, last_error, load, parareal_solve, to_params)

__all__ = ["BASKET", "CALL1", "CASH_OR_NOTHING", "COARSE_NUM", "COARSE_PINO", "EXCHANGE",
           "EXPORTS", "BSError", "Grid", "Pino", "bs_fine_sweeps", "bs_payoff",
           "coarse_propagate", "fine_propagate_batched", "last_error", "load", "parareal_solve",
           "to_params"]
