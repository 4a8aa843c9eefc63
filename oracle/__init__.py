"""FP64 CPU oracle for the sequential Metropolis Monte Carlo (arXiv:1602.05716).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline / reference legs import this package.  The product library never
does.  The C source (mco.c) cites the paper section each function follows.

Parity status: every function here is pinned by a CPU test against something
other than itself (cuRAND's host Philox stream, math.log, closed-form 2- and
3-ion energies, brute-force energy differences, the exact confined-pair
distance distribution, the ideal-gas limit and the Debye-Hueckel limiting law).  The delayed-acceptance part is
pinned by finite differences of the MLP gradient, libm's exp, brute-force features and near-field sums, exact
antisymmetry of the surrogate energy change, and the exact confined-pair distribution sampled by the
delayed-acceptance chain.  The energy autocorrelation (Sec. 5.2) is pinned by values derived by hand from its
definition, exact alternating series, affine invariance and the AR(1) closed form; the dressed-ion
analysis (Sec. 5.2) by the ideal gas (g = 1), synthetic far fields of known renormalised parameters and
the Debye-Hueckel limit.
"""
from .oracle import (OracleChain, build, lib, philox4x32_10, move_draws, log_L, total_energy,
                     RECORD_DTYPE, ACCEPT, REJECT_METROPOLIS, REJECT_OVERLAP, REJECT_WALL,
                     DA_REJECT1, DA_RECORD_DTYPE, MLP_NIN, MLP_H, MLP_NP, exp_D, bf16_to_f64, f64_to_bf16,
                     mlp_forward, mlp_loss_grad, energy_autocorr, dressed_ion_analysis,
                     pair_correlations)

__all__ = ["OracleChain", "build", "lib", "philox4x32_10", "move_draws", "log_L", "total_energy",
           "RECORD_DTYPE", "ACCEPT", "REJECT_METROPOLIS", "REJECT_OVERLAP", "REJECT_WALL",
           "DA_REJECT1", "DA_RECORD_DTYPE", "MLP_NIN", "MLP_H", "MLP_NP", "exp_D", "bf16_to_f64", "f64_to_bf16",
           "mlp_forward", "mlp_loss_grad", "energy_autocorr", "dressed_ion_analysis",
           "pair_correlations"]
