"""GB300-native sequential Metropolis Monte Carlo for primitive-model electrolytes.

Implements the hot path of Liang, Xing & Li (arXiv:1602.05716): exact O(N)
energy changes of sequential single-ion trial moves with hard-core overlap, a
hard spherical wall and the Metropolis test, as hand-written sm_103a CUDA
behind the C ABI of include/mc.h.  This package is a thin ctypes binding with
the same names; every step of the computation runs in the CUDA library, and
loading fails loudly when the library has not been built.
"""
from .api import (System, lib, build, device_info, test_philox, test_log, unit_rates, MCError, RECORD_DTYPE,
                  OPT_GUARD_MODE, OPT_TIMEOUT_MS, OPT_CTAS, OPT_SKIP_PUBLISH, OPT_USE_GRAPH, OPT_POLICY, OPT_DA, OPT_PAIRS, OPT_DEEP_WINDOWS, OPT_DRIFT_EVERY, OPT_HELPERS, OPT_DA_SWEEPS, OPT_SHARED_GUARD,
                  MLP_NIN, MLP_H, MLP_NP, mlp_forward, mlp_loss_grad, mlp_train, energy_autocorr, reduction_run, dressed_ion_analysis,
                  ERR_INVALID, ERR_OVERLAP_INIT, ERR_CUDA, ERR_TIMEOUT, ERR_OOM, ERR_POISONED)

__all__ = ["System", "lib", "build", "device_info", "test_philox", "test_log", "unit_rates", "MCError", "RECORD_DTYPE",
           "OPT_GUARD_MODE", "OPT_TIMEOUT_MS", "OPT_CTAS", "OPT_SKIP_PUBLISH", "OPT_USE_GRAPH", "OPT_POLICY", "OPT_DA", "OPT_PAIRS", "OPT_DEEP_WINDOWS", "OPT_DRIFT_EVERY", "OPT_HELPERS", "OPT_DA_SWEEPS", "OPT_SHARED_GUARD",
           "MLP_NIN", "MLP_H", "MLP_NP", "mlp_forward", "mlp_loss_grad", "mlp_train", "energy_autocorr", "reduction_run", "dressed_ion_analysis",
           "ERR_INVALID", "ERR_OVERLAP_INIT", "ERR_CUDA", "ERR_TIMEOUT", "ERR_OOM", "ERR_POISONED"]
