"""Bundle adjustment as a differentiable layer (torch.autograd.Function).

forward solves the problem with the C-ABI LM solver (mba_solve) and returns
the solved cameras and points; backward applies mba_adjoint at that solution,
giving the gradient with respect to the observations and the initial
estimate.  Argument marshalling only: the solve and the adjoint run in the
CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import mba


def _host(t: torch.Tensor, dtype=np.float64) -> np.ndarray:
    return np.ascontiguousarray(t.detach().to("cpu").numpy(), dtype=dtype)


class BALayer(torch.autograd.Function):
    """x* = argmin_x 1/2 sum rho(|pi(x) - u|^2) from the initial estimate x0.

    Inputs: observations (n, 2), cameras0 (nc, 9), points0 (np, 3), cam_idx (n,),
    pt_idx (n,), options (dict with ``precision``, ``loss``, ``huber_delta`` and
    solver options such as ``max_iter``, ``pcg_max_iter``, ``function_tol``;
    ``adjoint_mu``, ``adjoint_pcg_max_iter`` and ``adjoint_pcg_rel_tol`` control
    the backward solve; ``adjoint_mu`` < 0, the default, uses the damping of the
    last accepted LM step).  Outputs: cameras (nc, 9), points (np, 3), float64, on the
    observations' device.
    """

    @staticmethod
    def forward(ctx, observations, cameras0, points0, cam_idx, pt_idx, options=None):
        opts = dict(options or {})
        prob_kw = {k: opts.pop(k) for k in ("precision", "loss", "huber_delta") if k in opts}
        adj_kw = dict(pcg_max_iter=opts.pop("adjoint_pcg_max_iter", 500),
                      pcg_rel_tol=opts.pop("adjoint_pcg_rel_tol", 1e-12))
        ctx.adj_mu = float(opts.pop("adjoint_mu", -1.0))
        pr = mba.Problem(_host(cameras0), _host(points0), _host(observations), _host(cam_idx, np.int32),
                         _host(pt_idx, np.int32), **prob_kw)
        pr.solve(**opts)
        cams, pts = pr.parameters()
        ctx.problem, ctx.adj_kw, ctx.dev = pr, adj_kw, observations.device
        return (torch.from_numpy(cams).to(observations.device), torch.from_numpy(pts).to(observations.device))

    @staticmethod
    def backward(ctx, grad_cams, grad_pts):
        pr = ctx.problem
        if grad_cams is None:
            grad_cams = torch.zeros((pr.info["nc"], 9), dtype=torch.float64)
        if grad_pts is None:
            grad_pts = torch.zeros((pr.info["np"], 3), dtype=torch.float64)
        r = pr.adjoint(_host(grad_cams), _host(grad_pts), ctx.adj_mu, **ctx.adj_kw)
        pr.close()
        dev = ctx.dev
        return (torch.from_numpy(r["grad_obs"]).to(dev), torch.from_numpy(r["grad_init_cam"]).to(dev),
                torch.from_numpy(r["grad_init_pt"]).to(dev), None, None, None)


def ba_layer(observations, cameras0, points0, cam_idx, pt_idx, **options):
    """Functional form of BALayer."""
    return BALayer.apply(observations, cameras0, points0, cam_idx, pt_idx, options)
