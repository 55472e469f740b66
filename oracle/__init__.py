"""FP64 CPU oracle of the SQP / ADMM / implicit-differentiation OCP solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of the method, used to check the CUDA path.  Only `tests/`,
`__graft_entry__.smoke()` and the CPU-baseline / reference arm of `bench.py`
may import it; the product path (the C-ABI library and its Python binding)
never does, and it shares no code with it.

Modules (each function cites the passage of the paper it follows):
  models    dynamics f_t, constraints g_t and their Jacobians (Appendix A,
            Remark A1), centreline geometry of the racing model.
  qp        QP approximation at an SQP iterate (Section III-A, Appendix B):
            global sparse P, q, C, c, G and shifted bounds.
  admm      Algorithm 3 with the projection / smoothed projection of
            Section III-B, the residuals of Eq. (admm:residuals) and the
            adaptive rho rule of Eq. (rho:update).  The primal system
            S x = eta is formed as P + sigma I + A' rho A and solved by a
            library banded Cholesky (a plain definition, no block formulas).
            Optionally on the QP in normalised states and controls
            (problem rescaling, Remark 4).
  sqp       Algorithm 1 with the backtracking line search of Appendix D and
            the stopping test of Eq. (sqp_stop).
  backward  Algorithm 2: active set (Appendix E), the full active-set KKT
            system of Eq. (bwd:slack_adjoint) assembled sparse and solved by
            a library LU, and the vector-Jacobian product of Eq. (loss_gradient);
            optionally the reduced adjoint QP of Appendix E (hard active rows
            as penalties).

Parity status of each function is stated in its docstring; all of them are
pinned by `tests/test_oracle_*.py` except where a docstring says
"parity unpinned".
"""
