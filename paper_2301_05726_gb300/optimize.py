"""Variational optimisation of the UCC angles (the Methods section drives
them with SciPy's SLSQP; the paper does not say where its gradients come
from).

``minimize_energy`` takes any callable returning (E, dE/dtheta), so the same
driver runs on the GPU context (one adjoint sweep per evaluation) or on any
other implementation.  The optimiser itself is SciPy's.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import numpy as np


@dataclasses.dataclass
class OptResult:
    theta: np.ndarray
    energy: float
    grad_norm: float
    n_evals: int
    history: list
    success: bool
    message: str


def minimize_energy(energy_and_grad: Callable[[np.ndarray], tuple], theta0: np.ndarray, method: str = "SLSQP",
                    maxiter: int = 200, tol: float = 1e-10, callback: Optional[Callable] = None) -> OptResult:
    """Minimise E(theta) from theta0 with SciPy (SLSQP by default, as in the
    paper; L-BFGS-B and BFGS also work).  energy_and_grad(theta) -> (E, g)."""
    from scipy.optimize import minimize

    history = []
    cache = {}

    def fun(th):
        key = th.tobytes()
        if key not in cache:
            E, g = energy_and_grad(np.ascontiguousarray(th, dtype=np.float64))
            cache.clear()
            cache[key] = (float(E), np.array(g, dtype=np.float64))
            history.append(float(E))
            if callback is not None:
                callback(th, E, g)
        return cache[key]

    res = minimize(lambda th: fun(th)[0], np.asarray(theta0, dtype=np.float64), jac=lambda th: fun(th)[1],
                   method=method, tol=tol, options={"maxiter": maxiter})
    E, g = fun(res.x)
    return OptResult(theta=np.array(res.x), energy=E, grad_norm=float(np.linalg.norm(g)), n_evals=len(history),
                     history=history, success=bool(res.success), message=str(res.message))


def minimize_context(ctx, theta0: Optional[np.ndarray] = None, eps: Optional[float] = None, **kw) -> OptResult:
    """minimize_energy on a UCCContext: each evaluation uploads theta and runs
    apply + energy + the adjoint sweep on the GPU."""
    th0 = ctx.prob.theta if theta0 is None else theta0

    def eg(th):
        ctx.set_theta(th)
        return ctx.gradient(eps=eps)

    return minimize_energy(eg, th0, **kw)
