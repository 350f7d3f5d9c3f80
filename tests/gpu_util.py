"""Helpers shared by the GPU parity tests: upload a matgen CSR, build a plan
through the C ABI, compare against the oracle."""
import numpy as np

import oracle


def torch_dev():
    import torch
    return torch.device("cuda", 0)


def plan_for(A, **transform):
    """Analyze (and optionally transform) ``A`` through the C ABI."""
    from paper_2103_11445_gb300 import binding as B
    P = B.Plan(A.n, A.row_ptr, A.col, A.val)
    if transform:
        P.transform(**transform)
    return P


def gpu_solve(P, b):
    import torch
    bt = torch.as_tensor(np.ascontiguousarray(b), device=torch_dev())
    x = P.solve(bt)
    P.check()
    return x.cpu().numpy()


def assert_close_to_oracle(A, x, b, tol):
    ref = oracle.forward_subst(A, b)
    err = oracle.relerr(x, ref)
    assert err <= tol, f"relerr {err:.3e} > {tol:.1e}"
    return err
