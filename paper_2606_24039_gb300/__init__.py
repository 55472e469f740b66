"""GB300-native batched differentiable MPC: SQP with an ADMM QP solver whose
block-tridiagonal primal system is factored once per SQP step / rho change,
and an active-set implicit-differentiation backward pass (arxiv 2606.24039).

The compute path is the CUDA library behind the C ABI of include/tmpc.h
(built by `build.build()`); this package only marshals arguments to it.
"""
from ._abi import TmpcError, default_options, load  # noqa: F401
from .solver import (Solver, TmpcFunction, options_from, solve_ocp, tensors_from_batch,  # noqa: F401
                     tmpc_solve_static)
