"""torch.autograd binding of the differentiable hopping score.

``score_points`` evaluates the continuous-point score of gh_score_points
(both map axes polar-interpolated) and differentiates it through
gh_score_points_adjoint with respect to the points (x, y, vx, vy), the
receiver positions and the complex64 maps. Argument marshalling only: the
forward and backward passes run in the library's kernels.
"""
from __future__ import annotations

import torch

from . import gh


class _ScorePoints(torch.autograd.Function):
    @staticmethod
    def forward(fctx, maps, points, rx, lib, radar, tx, map_dtype):
        P = points.shape[0]
        S = torch.empty(P, dtype=torch.float32, device=points.device)
        lib.gh_score_points(radar, tx, rx, rx.shape[0], maps, points, P, S, map_dtype=map_dtype)
        fctx.save_for_backward(maps, points, rx)
        fctx.lib, fctx.radar, fctx.tx, fctx.map_dtype = lib, radar, tx, map_dtype
        return S

    @staticmethod
    def backward(fctx, gS):
        maps, points, rx = fctx.saved_tensors
        need_maps, need_points, need_rx = fctx.needs_input_grad[:3]
        gS = gS.contiguous().to(torch.float32)
        dpoints = torch.empty_like(points) if need_points else None
        drx = torch.zeros_like(rx) if need_rx else None
        dmaps = torch.zeros_like(maps) if need_maps else None
        fctx.lib.gh_score_points_adjoint(fctx.radar, fctx.tx, rx, rx.shape[0], maps, points, points.shape[0], gS,
                                         dpoints, drx, dmaps, map_dtype=fctx.map_dtype)
        return dmaps, dpoints, drx, None, None, None, None


def score_points(lib: gh.Context, radar, tx, rx: torch.Tensor, maps: torch.Tensor, points: torch.Tensor):
    """Scores (float32 [P]) of the points (float64 [P, 4] on the device) with
    receivers at rx (float64 [Q, 2] on the device); differentiable with
    respect to points, rx and (complex64) maps."""
    if points.dtype != torch.float64 or points.dim() != 2 or points.shape[1] != 4:
        raise ValueError("points must be float64 [P, 4]")
    if rx.dtype != torch.float64 or rx.dim() != 2 or rx.shape[1] != 2:
        raise ValueError("rx must be float64 [Q, 2]")
    map_dtype = gh.Context.map_dtype_of(maps)
    if maps.requires_grad and map_dtype != gh.GH_C64:
        raise ValueError("map gradients need complex64 maps")
    return _ScorePoints.apply(maps, points.contiguous(), rx.contiguous(), lib, radar, tx, map_dtype)


def refine(lib: gh.Context, radar, tx, rx: torch.Tensor, maps: torch.Tensor, points: torch.Tensor, iters: int = 20,
           scale_xy: float = 0.3, scale_v: float = 1.0, step: float = 0.5):
    """Off-grid refinement of detections by damped Newton ascent of the score
    (one launch, gh_refine_points). Returns (refined points, their scores)."""
    out = points.detach().clone().contiguous()
    S = torch.empty(out.shape[0], dtype=torch.float32, device=out.device)
    lib.gh_refine_points(radar, tx, rx.detach().contiguous(), rx.shape[0], maps, out, out.shape[0], iters, scale_xy,
                         scale_v, step, S, map_dtype=gh.Context.map_dtype_of(maps))
    return out, S
