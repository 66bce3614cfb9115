"""Densification, pruning and opacity reset (through the C ABI) against the
oracle (oracle/densify.py): the decisions and counts bit for bit, surviving
and cloned rows as exact copies, children's means within float32 rounding
and their log-scales exactly, Adam moments / freeze map / extra state
carried or zeroed; the projection backward's second statistics window."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import densify as D  # noqa: E402
from paper_2504_06716_gb300 import lib, synth  # noqa: E402

import parity_util as pu  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    oracle.build()
    lib.load()


def _prm(prune_big, use_rgb, extent=4.4):
    p = D.DensifyParams(eps_xyz=float(np.float32(2e-4)), eps_rgb=float(np.float32(1e-6)), use_rgb=use_rgb,
                        log_clone_max=float(np.float32(math.log(0.01 * extent))),
                        logit_min_opacity=float(np.float32(D.logit(0.005))), prune_big=prune_big,
                        max_screen_radius=20, log_max_world=float(np.float32(math.log(0.1 * extent))),
                        log_split_div=float(np.float32(math.log(1.6))))
    g = lib.GsDensifyParams(p.eps_xyz, p.eps_rgb, int(p.use_rgb), p.log_clone_max, p.logit_min_opacity,
                            int(p.prune_big), p.max_screen_radius, p.log_max_world, p.log_split_div)
    return p, g


def _case(n, seed):
    g = np.random.default_rng(seed)
    P = synth.gaussians_surface(n, seed)
    P[:, 3:6] += g.normal(0.0, 1.2, (n, 3))              # scales from tiny to too big
    P[:, 10] = g.normal(-1.0, 3.0, n)                      # some below logit(0.005)
    P = pu.f32(P)
    cnt = g.integers(0, 6, n).astype(np.int32)
    acc_x = (g.exponential(1.5e-4, n) * cnt).astype(np.float32)
    acc_r = (g.exponential(8e-7, n) * cnt).astype(np.float32)
    maxr = g.integers(0, 40, n).astype(np.int32)
    return P, acc_x, acc_r, cnt, maxr


def _gpu(P, acc_x, acc_r, cnt, maxr, gprm, z_for=None, capacity=None, extra_w=3, seed=0):
    n = P.shape[0]
    g = np.random.default_rng(seed + 99)
    t = lambda a, dt=torch.float32: torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dt)  # noqa: E731
    Pt = t(pu.pack64(P))
    m = t(g.normal(0, 1e-3, (n, 64)).astype(np.float32))
    v = t(g.uniform(0, 1e-4, (n, 64)).astype(np.float32))
    frozen = t((g.uniform(size=n) < 0.3).astype(np.uint8), torch.uint8)
    extra = t(g.normal(0, 1, (n, extra_w)).astype(np.float32))
    st_t = (t(acc_x), t(acc_r), t(cnt, torch.int32), t(maxr, torch.int32))  # kept alive: the struct holds pointers
    stats = lib.grad_stats(*st_t)
    ws = torch.zeros(lib.gs_densify_workspace_bytes(n), dtype=torch.uint8, device=DEV)
    counts = torch.zeros(4, dtype=torch.int64, device=DEV)
    lib.gs_densify_plan(n, Pt, stats, gprm, ws, counts)
    c = counts.cpu().numpy()
    n_out = int(c[0] + c[1] + c[2])
    z = z_for(int(c[3])) if z_for else np.zeros((int(c[3]), 2, 3), np.float32)
    cap = n_out if capacity is None else capacity
    outs = [torch.full((max(cap, 1), 64), -5.0, device=DEV) for _ in range(3)]
    fo = torch.full((max(cap, 1),), 7, dtype=torch.uint8, device=DEV)
    eo = torch.full((max(cap, 1), extra_w), -5.0, device=DEV)
    cnt_t = t(cnt, torch.int32)
    co = torch.full((max(cap, 1),), -5, dtype=torch.int32, device=DEV)
    carries = [lib.densify_carry(extra, eo), lib.densify_carry(cnt_t, co)] if n else []
    lib.gs_densify_apply(n, Pt, m, v, frozen, carries, gprm,
                         t(z.astype(np.float32)) if z.size else torch.zeros(1, device=DEV), ws, cap, outs[0], outs[1],
                         outs[2], fo)
    assert lib.gs_get_device_error() == 0
    return dict(counts=c, n_out=n_out, P=outs[0].cpu().numpy(), m=outs[1].cpu().numpy(), v=outs[2].cpu().numpy(),
                frozen=fo.cpu().numpy(), extra=eo.cpu().numpy(), m_in=m.cpu().numpy(), v_in=v.cpu().numpy(),
                frozen_in=frozen.cpu().numpy(), extra_in=extra.cpu().numpy(), cnt_out=co.cpu().numpy(), z=z)


@pytest.mark.parametrize("prune_big,use_rgb,n", [(False, False, 50001), (True, True, 50001), (True, False, 1)])
def test_densify_matches_oracle(prune_big, use_rgb, n):
    P, ax, ar, cnt, maxr = _case(n, 3 + n)
    p, gp = _prm(prune_big, use_rgb)
    zg = np.random.default_rng(17)
    res = _gpu(P, ax, ar, cnt, maxr, gp, z_for=lambda k: zg.standard_normal((k, 2, 3)).astype(np.float32))
    want = D.densify(P, ax, ar, cnt, maxr, p, res["z"].astype(np.float64))
    wc = want["counts"]
    assert res["counts"].tolist() == [wc["kept"], wc["clones"], wc["children"], wc["splits"]]
    k = res["n_out"]
    assert k == len(want["src"])
    src, kind = want["src"], want["kind"]
    got = res["P"][:k, :59].astype(np.float64)
    new = kind != 0
    # rows copied exactly: survivors, clones, and the children's untouched parameters
    assert np.array_equal(got[kind <= 1], want["P"][kind <= 1])
    assert np.array_equal(got[kind >= 2][:, 6:], want["P"][kind >= 2][:, 6:])
    assert np.array_equal(got[kind >= 2][:, 3:6], want["P"][kind >= 2][:, 3:6])  # float32 log-scale shift
    # children's means: float32 arithmetic against double
    if (kind >= 2).any():
        scale = np.abs(want["P"][kind >= 2][:, 0:3]) + np.exp(P[src[kind >= 2], 3:6].max(axis=1))[:, None] * 6
        assert np.all(np.abs(got[kind >= 2][:, 0:3] - want["P"][kind >= 2][:, 0:3]) <= 2e-6 * scale)
    # state carried for survivors, zero / unfrozen for new Gaussians
    assert np.array_equal(res["m"][:k][~new], res["m_in"][src[~new]])
    assert np.array_equal(res["v"][:k][~new], res["v_in"][src[~new]])
    assert not res["m"][:k][new].any() and not res["v"][:k][new].any()
    assert np.array_equal(res["frozen"][:k], D.carry(res["frozen_in"], src, kind, 0))
    assert np.array_equal(res["extra"][:k], D.carry(res["extra_in"], src, kind, 0.0))
    assert np.array_equal(res["cnt_out"][:k], D.carry(cnt, src, kind, 0))  # an int32 array carried too
    if n > 1:
        assert wc["clones"] > 0 and wc["splits"] > 0 and wc["kept"] < n  # every outcome happens


def test_densify_empty_and_all_pruned_and_small_capacity():
    p, gp = _prm(False, False)
    ws = torch.zeros(lib.gs_densify_workspace_bytes(0), dtype=torch.uint8, device=DEV)
    counts = torch.full((4,), 9, dtype=torch.int64, device=DEV)
    one, ione = torch.zeros(1, device=DEV), torch.zeros(1, dtype=torch.int32, device=DEV)
    lib.gs_densify_plan(0, one, lib.grad_stats(one, one, ione), gp, ws, counts)
    assert counts.cpu().tolist() == [0, 0, 0, 0]
    P, ax, ar, cnt, maxr = _case(2000, 5)
    P[:, 10] = -12.0  # everything below the opacity floor
    res = _gpu(P, ax, ar, cnt, maxr, gp)
    assert res["n_out"] == 0
    P, ax, ar, cnt, maxr = _case(2000, 6)
    res = _gpu(P, ax, ar, cnt, maxr, gp, capacity=10)  # too small: nothing written
    assert res["n_out"] > 10 and np.all(res["P"][:10] == -5.0)


def test_opacity_reset_matches_oracle():
    g = np.random.default_rng(8)
    n = 10007
    P = g.normal(0, 3, (n, 64)).astype(np.float32)
    M, V = g.normal(0, 1, (n, 64)).astype(np.float32), g.uniform(0, 1, (n, 64)).astype(np.float32)
    cap = float(np.float32(D.logit(0.01)))
    frozen = (g.uniform(size=n) < 0.3).astype(np.uint8)
    for fr in (None, frozen):
        P2, M2, V2 = P.copy(), M.copy(), V.copy()
        t = [torch.from_numpy(a.copy()).to(DEV) for a in (P2, M2, V2)]
        lib.gs_opacity_reset(n, t[0], t[1], t[2], cap, None if fr is None else torch.from_numpy(fr).to(DEV))
        D.opacity_reset(P2, M2, V2, cap, fr)
        assert np.array_equal(t[0].cpu().numpy(), P2) and np.array_equal(t[1].cpu().numpy(), M2)
        assert np.array_equal(t[2].cpu().numpy(), V2)
        if fr is not None:  # frozen rows untouched
            assert np.array_equal(P2[fr == 1], P[fr == 1]) and np.array_equal(M2[fr == 1], M[fr == 1])


def test_projection_backward_updates_two_statistics_windows():
    n = 20000
    P = pu.f32(synth.gaussians_surface(n, 31))
    Pt = torch.from_numpy(pu.pack64(P)).to(DEV)
    cam = lib.camera(synth.hemisphere_cameras(2, 4.0, 320, 240, 60.0)[1], tile=16)
    spl = torch.zeros((n, 12), device=DEV)
    lib.gs_project(Pt, n, 3, cam, spl)
    act = torch.arange(0, n, 2, dtype=torch.int32, device=DEV)
    na = torch.tensor([act.numel()], dtype=torch.int32, device=DEV)
    g2 = torch.from_numpy(np.random.default_rng(32).normal(0, 1e-4, (n, 12)).astype(np.float32)).to(DEV)
    z = lambda dt=torch.float32: torch.zeros(n, dtype=dt, device=DEV)  # noqa: E731
    a1 = (z(), z(), z(torch.int32))
    a2 = (z(), z(), z(torch.int32), torch.full((n,), 3, dtype=torch.int32, device=DEV))
    G1, G2 = torch.zeros((n, 64), device=DEV), torch.zeros((n, 64), device=DEV)
    lib.gs_project_bwd(Pt, n, 3, cam, spl, act, na, g2.clone(), G1, *a1)
    lib.gs_project_bwd_stats(Pt, n, 3, cam, spl, act, na, g2.clone(), G2, False, [lib.grad_stats(*a2[:3], a2[3])])
    assert torch.equal(G1, G2)
    for x, y in zip(a1, a2[:3]):
        assert torch.equal(x, y)
    rad = spl[:, 10].contiguous().view(torch.int32)
    want = torch.full((n,), 3, dtype=torch.int32, device=DEV)
    touched = torch.zeros(n, dtype=torch.bool, device=DEV)
    touched[act.long()] = True
    vis = touched & (rad > 0)
    want[vis] = torch.maximum(want[vis], rad[vis])
    assert torch.equal(a2[3], want)
    # two windows at once: both get the same increments
    b1, b2 = (z(), z(), z(torch.int32)), (z(), z(), z(torch.int32))
    lib.gs_project_bwd_stats(Pt, n, 3, cam, spl, act, na, g2.clone(), G2, False,
                             [lib.grad_stats(*b1), lib.grad_stats(*b2)])
    for x, y, w in zip(b1, b2, a1):
        assert torch.equal(x, y) and torch.equal(x, w)
