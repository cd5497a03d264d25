"""Gradients of the FP64 oracle (TEST INFRASTRUCTURE).

The paper optimises splat positions, rotations, scales, opacities, the
material texture maps and the environment maps end to end (Sec. 3.6).  The
reference gradient here is the exact derivative of the FP64 forward of
render.py, taken by torch autograd (a library primitive applied to the plain
definition), of the scalar  S = sum(rgba * dL_drgba)  for a given upstream
gradient image.  Discrete decisions (support cut, alpha threshold and clamp,
termination, texel/face/level index choice, orientation flip, culling and the
depth order) carry zero derivative; derivatives through bilinear weights,
LUT and cube coordinates are kept.

Parity: pinned against central finite differences of the same forward
(tests/test_oracle_grad.py).
"""
from __future__ import annotations

import numpy as np
import torch

from . import render as R

PARAM_NAMES = ("means", "quats", "scales", "opacity", "texels")


def render_grads(scene: dict, cam: dict, env: dict, dL_drgba: np.ndarray, *, tiles=None,
                 keylist=None, max_entries=2_000_000, normal_weight: float = 0.0, vis=None) -> dict:
    """Autograd gradients of sum(rgba * dL_drgba) w.r.t. every parameter.

    With ``normal_weight`` the objective adds normal_weight x L_n (the
    normal-consistency loss of oracle/loss.py over the whole view).
    Returns numpy float64 arrays for means, quats, scales, opacity, texels,
    spec (list per level) and irr, plus the rendered rgba.
    """
    params = R.to_params(scene, requires_grad=True)
    envp = R.env_params(env, requires_grad=True)
    g = torch.from_numpy(np.asarray(dL_drgba, dtype=np.float64))
    out = R.render(scene, cam, env, params=params, envp=envp, tiles=tiles, margins=None,
                   max_entries=max_entries, keylist=keylist, vis=vis)
    S = (out["rgba"] * g).sum()
    if normal_weight:
        from .loss import depth_normal_loss
        Ln, _, _ = depth_normal_loss(out["Z"], out["A"], out["X"], cam)
        S = S + normal_weight * Ln
    S.backward()
    res = {k: params[k].grad.numpy().copy() for k in PARAM_NAMES}
    if "sh" in params:
        res["sh"] = params["sh"].grad.numpy().copy()
    res["spec"] = [m.grad.numpy().copy() for m in envp["spec"]]
    res["irr"] = envp["irr"].grad.numpy().copy()
    res["rgba"] = out["rgba"].detach().numpy()
    return res


def scalar_objective(scene: dict, cam: dict, env: dict, dL_drgba: np.ndarray, keylist=None, vis=None) -> float:
    """S = sum(rgba * dL_drgba) of the FP64 forward (for finite differences).

    The key list (tile binning, culling, order) is held fixed by passing the
    unperturbed one, so a difference quotient sees only the smooth part."""
    out = R.render(scene, cam, env, margins=None, keylist=keylist, vis=vis)
    return float((out["rgba"] * torch.from_numpy(np.asarray(dL_drgba, dtype=np.float64))).sum())


def central_difference(scene: dict, cam: dict, env: dict, dL_drgba, name: str, index, h: float,
                       keylist=None, vis=None) -> float:
    """(S(x + h e) - S(x - h e)) / 2h for one parameter entry.  ``name`` is a
    scene key, or ('spec', level) / 'irr' for the environment maps.  Values
    are perturbed in float64 copies (no float32 rounding of the step)."""
    def perturbed(sign):
        sc = {k: (np.asarray(v, dtype=np.float64).copy() if isinstance(v, np.ndarray) else v)
              for k, v in scene.items()}
        ev = dict(env, spec=[np.asarray(m, dtype=np.float64).copy() for m in env["spec"]],
                  irr=np.asarray(env["irr"], dtype=np.float64).copy())
        if isinstance(name, tuple) and name[0] == "spec":
            ev["spec"][name[1]][index] += sign * h
        elif name == "irr":
            ev["irr"][index] += sign * h
        else:
            sc[name][index] += sign * h
        return scalar_objective(sc, cam, ev, dL_drgba, keylist=keylist, vis=vis)

    return (perturbed(+1.0) - perturbed(-1.0)) / (2.0 * h)
