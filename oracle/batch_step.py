"""One training step of several scenes at once, written out plainly (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper trains one scene on one view per iteration (Algorithm 1). The
batched workload (several scenes of uneven size, several views of each per
step) is not in the paper; its reading, stated here and applied by the CUDA
path as well:

* a scene's step starts with the freeze-map action of Algorithm 1 for that
  iteration (Eqs. 4-6 on the statistics gathered since the previous
  boundary; thresholds from Eq. 5), decided on the scene's own map;
* each of the scene's views is rendered and differentiated on that map
  (Eq. 2, Eq. 3, frozen Gaussians get no gradient, Sec. 3.2.4);
* the scene's gradient is the sum of its views' gradients;
* the freeze statistics count each view in which a Gaussian is visible and
  unfrozen as one visibility, adding that view's norms (Eq. 4's averages);
* one masked Adam step per scene (Sec. 3.2.4), its bias correction taken at
  the scene's own step counter, which advances by one per batch step.

Each scene is independent of the others: the batch changes how the work is
launched, not what a scene computes.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import planted


def scene_step(P, M, V, frozen, acc_x, acc_r, cnt, cams, gts, lr, step: int, b1: float = 0.9, b2: float = 0.999,
               eps: float = 1e-15, sh_degree: int = 3, smooth: bool = False) -> dict:
    """The views' part and the optimiser step of one scene, in place on float64
    P, M, V [n][59] and float64 statistics acc_x, acc_r, int cnt [n]. ``frozen``
    is the map after the step's freeze action. Returns the summed gradient G,
    each view's loss and forward. ``smooth`` drops the cut-offs (for finite
    differences)."""
    n = P.shape[0]
    G = np.zeros((n, oracle.N_PARAMS))
    losses, fwds = [], []
    for cam, gt in zip(cams, gts):
        res = oracle.loss_and_grad(P, cam, gt, frozen=frozen, sh_degree=sh_degree, smooth=smooth)
        G += res["G"]
        live = (res["fwd"]["proj"]["radius"] > 0) & (frozen == 0)
        acc_x[live] += res["xyz_norm"][live]
        acc_r[live] += res["rgb_norm"][live]
        cnt[live] += 1
        losses.append(res["loss"])
        fwds.append(res)
        if planted(46):  # the last view alone
            G = res["G"].copy()
    oracle.adam(P, G, M, V, frozen, lr, step + (1 if planted(47) else 0), b1, b2, eps)
    return dict(G=G, losses=losses, views=fwds)


def batch_step(scenes: list[dict], k: int, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-15) -> list[dict]:
    """Iteration k for every scene of the batch. Each scene is a dict with P,
    M, V (float64 [n][59]), frozen (uint8 [n]), acc_x, acc_r (float32 [n]),
    cnt (int32 [n]), step (its Adam step count so far), lr (6 group rates),
    cams and gts (its views in this step), and ``action``: the freeze-map
    mode of Algorithm 1 for k (0 update, 1 reset, 2 restart the statistics,
    None nothing) with its thresholds ``eps_xyz``, ``eps_rgb``. Updated in
    place; returns each scene's step result with its active list."""
    out = []
    for s in scenes:
        act = None
        if s["action"] is not None:
            act = oracle.freeze_update(s["acc_x"], s["acc_r"], s["cnt"], s["frozen"], s["eps_xyz"], s["eps_rgb"],
                                       s["action"])
        ax = s["acc_x"].astype(np.float64)
        ar = s["acc_r"].astype(np.float64)
        c = s["cnt"].astype(np.int64)
        s["step"] += 1
        res = scene_step(s["P"], s["M"], s["V"], s["frozen"], ax, ar, c, s["cams"], s["gts"], s["lr"], s["step"], b1,
                         b2, eps)
        s["acc_x"], s["acc_r"], s["cnt"] = ax, ar, c
        res["act"] = act
        out.append(res)
    return out
