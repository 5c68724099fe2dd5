"""Joint estimation of per-view geometry drift and the image (the paper's
motivation in Sec. 1: a scan whose source and detector drift during the
acquisition is reconstructed while the drift is estimated).

Alternation, coarse grids first:
  * the image step: multigrid iterations of Alg. 1 with the current drift
    estimate set on the geometry;
  * the drift step: per-view Newton steps on phi_k = (ds_u, ds_v, dd_u,
    dd_v, psi) for the loss 1/2 |A(phi) mu - b|^2 on grid `level`, with mu
    the current image restricted to that grid.  The views decouple (view k's
    residual depends on phi_k alone), so the Hessian is 5 x 5 per view; its
    columns come from differences of the library's geometry gradient
    (mgct_geometry_grad, the adjoint kernel of the differentiable form)
    under a small step of one parameter type in every view at once.  A
    Levenberg-Marquardt damping and a trust region (one pixel of the grid)
    keep the steps safe where the data pin a parameter weakly (a source and
    a detector shift along the same axis move the projections alike, up to
    the magnification across the volume's depth).

Every operator is one of the library's: the projector, the geometry gradient,
restriction and the multigrid iteration.  The host solves the 5 x 5 systems.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mgct


def _restrict_to(x: torch.Tensor, level: int, fn) -> torch.Tensor:
    for _ in range(level):
        x = fn(x)
    return x


def newton_drift_step(geom, mu_l: torch.Tensor, b_l: torch.Tensor, phi: np.ndarray, level: int,
                      half_diag_px: float, damping: float = 1e-2) -> tuple[np.ndarray, float]:
    """One damped Newton step on every view's drift at grid `level`; returns
    (new phi, loss before the step)."""
    K = phi.shape[0]
    eps = np.array([0.05, 0.05, 0.05, 0.05, 0.05 / max(half_diag_px, 1.0)])

    def grad_at(p):
        geom.set_drift(p)
        neg_r = mgct.project(geom, mu_l, level=level, b=b_l)  # b - A mu
        r = -neg_r
        gk = mgct.geometry_grad(geom, mu_l, r, level=level)
        loss = 0.5 * float((neg_r.double() ** 2).sum())
        return gk.cpu().numpy(), loss

    g0, loss = grad_at(phi)
    H = np.empty((K, 5, 5))
    for j in range(5):
        p = phi.copy()
        p[:, j] += eps[j]
        gj, _ = grad_at(p)
        H[:, :, j] = (gj - g0) / eps[j]
    H = 0.5 * (H + np.transpose(H, (0, 2, 1)))
    diag = np.abs(np.diagonal(H, axis1=1, axis2=2)) + 1e-30
    A = H + damping * diag[:, :, None] * np.eye(5)[None]
    try:
        step = -np.linalg.solve(A, g0[:, :, None])[:, :, 0]
    except np.linalg.LinAlgError:
        step = -g0 / diag
    # trust region: one pixel of this grid (and the matching tilt)
    lim = np.array([1.0, 1.0, 1.0, 1.0, 1.0 / max(half_diag_px, 1.0)]) * (1 << level)
    step = np.clip(step, -lim, lim)
    geom.set_drift(phi)
    return phi + step, loss


def estimate(geom, b: torch.Tensor, half_diag_px: float, schedule=((1, 2), (0, 2)), mg_iters: int = 2,
             newton_steps: int = 2, phi0: np.ndarray | None = None, truth_phi: np.ndarray | None = None,
             mu: torch.Tensor | None = None):
    """Alternate image and drift steps.  `schedule` lists (grid, rounds);
    each round runs `mg_iters` multigrid iterations, then `newton_steps`
    drift steps on that grid.  Returns (mu, phi, history); with `truth_phi`
    the history records the drift RMSE per parameter type after each round."""
    K = geom.n_views
    phi = np.zeros((K, 5)) if phi0 is None else np.array(phi0, dtype=np.float64)
    n = geom.n
    if mu is None:
        mu = torch.zeros((n, n, n), device=b.device, dtype=torch.float32)
    rec = mgct.Reconstructor(geom)
    hist = []
    for level, rounds in schedule:
        b_l = _restrict_to(b, level, mgct.restrict_sino)
        for _ in range(rounds):
            geom.set_drift(phi)
            rec.prepare(b)
            for _ in range(mg_iters):
                rec.iterate(mu)
            mu_l = _restrict_to(mu, level, mgct.restrict_volume).contiguous()
            loss = None
            for _ in range(newton_steps):
                phi, loss = newton_drift_step(geom, mu_l, b_l, phi, level, half_diag_px)
            rec_h = {"level": level, "loss_before_last_step": loss}
            if truth_phi is not None:
                rec_h["drift_rmse"] = np.sqrt(np.mean((phi - truth_phi) ** 2, axis=0)).tolist()
            hist.append(rec_h)
    geom.set_drift(phi)
    rec.prepare(b)
    for _ in range(mg_iters):
        rec.iterate(mu)
    return mu, phi, hist
