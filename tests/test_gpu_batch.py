"""The batched path for several scenes of uneven size (through the C ABI):

* one persistent launch over many (scene, view) jobs gives, job by job, what
  the single-job rasteriser gives (the forward bit for bit; the backward up to
  the order of its float atomics), for every tile size, on ragged images;
  jobs of one scene may share a gradient buffer; a job with a mismatched
  camera is skipped and flagged;
* gs_project_bwd_accum adds exactly what gs_project_bwd writes;
* the device-step Adam equals the host-step Adam;
* the CUDA-graph replay of a batch step trains like the eager step and like
  one launch per job, scenes finish and leave the batch, and the autotuner
  returns a working launch shape.

The single-job kernels these are compared with are checked against the FP64
oracle in test_gpu_parity.py and test_gpu_e2e.py.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
    lib.load()


W, H = 200, 152  # ragged for every tile size


def _jobs_setup(tile, seed=0):
    """Three scenes of uneven size, two views each: per job the projected
    splats, sorted lists, a seeded image gradient; per scene a frozen map."""
    sizes = (3000, 15000, 40000)
    jobs = []
    for si, n in enumerate(sizes):
        P = pu.f32(synth.gaussians_surface(n, seed + si))
        Pt = torch.from_numpy(pu.pack64(P)).to(DEV)
        frozen = torch.from_numpy((np.random.default_rng(seed + 10 + si).uniform(size=n) < 0.25).astype(np.uint8)).to(
            DEV)
        for vi, c in enumerate(synth.hemisphere_cameras(2, 4.0, W, H, 60.0)):
            cam = lib.camera(c, tile=tile)
            spl = torch.zeros((n, 12), dtype=torch.float32, device=DEV)
            lib.gs_project(Pt, n, 3, cam, spl)
            cap = int(spl[:, 11].contiguous().view(torch.int32).to(torch.int64).sum().item()) + 64
            ws = torch.zeros(lib.gs_sort_workspace_bytes(n, cap, cam), dtype=torch.uint8, device=DEV)
            vals = torch.zeros(cap, dtype=torch.int32, device=DEV)
            ranges = torch.zeros((cam.tiles, 2), dtype=torch.int32, device=DEV)
            count = torch.zeros(1, dtype=torch.int64, device=DEV)
            lib.gs_sort(spl, n, cam, ws, cap, vals, ranges, count)
            g = torch.Generator(device="cpu").manual_seed(seed * 100 + si * 10 + vi)
            dl = (torch.randn((3, H, W), generator=g) * 1e-3).to(DEV)
            jobs.append(dict(scene=si, n=n, cam=cam, splats=spl, vals=vals, ranges=ranges, dl=dl, frozen=frozen))
    return jobs


def _out_bufs(j):
    return dict(image=torch.full((3, H, W), -7.0, device=DEV), t_final=torch.full((H, W), -7.0, device=DEV),
                n_last=torch.full((H, W), -7, dtype=torch.int32, device=DEV),
                grad2d=torch.zeros((j["n"], 12), dtype=torch.float32, device=DEV))


def _table(jobs, outs, cams=None):
    recs = []
    for i, (j, o) in enumerate(zip(jobs, outs)):
        recs.append(lib.GsRasterJob(j["splats"].data_ptr(), j["vals"].data_ptr(), j["ranges"].data_ptr(),
                                    o["image"].data_ptr(), o["t_final"].data_ptr(), o["n_last"].data_ptr(),
                                    j["dl"].data_ptr(), j["frozen"].data_ptr(), o["grad2d"].data_ptr(),
                                    (cams or {}).get(i, j["cam"])))
    raw = (lib.GsRasterJob * len(recs))(*recs)
    return torch.frombuffer(bytearray(bytes(raw)), dtype=torch.uint8).to(DEV)


def _grad_close(got, want):
    """Same terms summed in another order by float atomics."""
    scale = want.abs().amax(dim=0, keepdim=True).clamp(min=1e-30)
    return bool(((got - want).abs() <= 1e-5 * (got.abs() + want.abs()) + 1e-6 * scale).all())


@pytest.mark.parametrize("tile,cfg", [(8, None), (8, (2, 32)), (16, None), (16, (1, 128)), (32, None), (32, (2, 256))])
def test_batch_launch_matches_single_job_launches(tile, cfg):
    jobs = _jobs_setup(tile)
    c = None if cfg is None else lib.raster_config(*cfg)
    ref = [_out_bufs(j) for j in jobs]
    for j, o in zip(jobs, ref):
        lib.gs_render_fwd_cfg(j["splats"], j["vals"], j["ranges"], j["cam"], c, o["image"], o["t_final"], o["n_last"])
        lib.gs_raster_bwd_cfg(j["splats"], j["vals"], j["ranges"], j["cam"], c, o["t_final"], o["n_last"], j["dl"],
                              j["frozen"], o["grad2d"])
    out = [_out_bufs(j) for j in jobs]
    table = _table(jobs, out)
    queue = torch.zeros(1, dtype=torch.int32, device=DEV)
    lib.gs_render_fwd_batch(table, len(jobs), W, H, tile, c, queue)
    lib.gs_raster_bwd_batch(table, len(jobs), W, H, tile, c, queue)
    assert lib.gs_get_device_error() == 0
    for j, o, r in zip(jobs, out, ref):
        assert torch.equal(o["image"], r["image"]) and torch.equal(o["t_final"], r["t_final"])
        assert torch.equal(o["n_last"], r["n_last"])
        assert _grad_close(o["grad2d"], r["grad2d"])
        assert not o["grad2d"][j["frozen"].bool()].any()  # frozen Gaussians get nothing
    assert int(queue.item()) >= len(jobs) * jobs[0]["cam"].tiles  # every item was taken


def test_jobs_of_one_scene_share_a_gradient_buffer():
    jobs = [j for j in _jobs_setup(16, seed=3) if j["scene"] == 2]
    single = []
    for j in jobs:
        o = _out_bufs(j)
        lib.gs_render_fwd(j["splats"], j["vals"], j["ranges"], j["cam"], o["image"], o["t_final"], o["n_last"])
        lib.gs_raster_bwd(j["splats"], j["vals"], j["ranges"], j["cam"], o["t_final"], o["n_last"], j["dl"],
                          j["frozen"], o["grad2d"])
        single.append(o)
    outs = [_out_bufs(j) for j in jobs]
    outs[1]["grad2d"] = outs[0]["grad2d"]
    table = _table(jobs, outs)
    queue = torch.zeros(1, dtype=torch.int32, device=DEV)
    lib.gs_render_fwd_batch(table, len(jobs), W, H, 16, None, queue)
    lib.gs_raster_bwd_batch(table, len(jobs), W, H, 16, None, queue)
    assert _grad_close(outs[0]["grad2d"], single[0]["grad2d"] + single[1]["grad2d"])


def test_mismatched_job_is_skipped_and_flagged():
    jobs = _jobs_setup(16, seed=5)[:2]
    outs = [_out_bufs(j) for j in jobs]
    bad = lib.camera(synth.hemisphere_cameras(2, 4.0, W, H, 60.0)[1], tile=8)  # wrong tile for a tile-16 batch
    table = _table(jobs, outs, cams={1: bad})
    queue = torch.zeros(1, dtype=torch.int32, device=DEV)
    lib.gs_render_fwd_batch(table, 2, W, H, 16, None, queue)
    flags = lib.gs_get_device_error()
    assert flags & lib.GS_FLAG_BADJOB
    assert bool((outs[1]["image"] == -7.0).all())  # untouched
    ref = _out_bufs(jobs[0])
    j = jobs[0]
    lib.gs_render_fwd(j["splats"], j["vals"], j["ranges"], j["cam"], ref["image"], ref["t_final"], ref["n_last"])
    assert torch.equal(outs[0]["image"], ref["image"])
    assert lib.gs_get_device_error() == 0  # the flag was cleared by the read


def test_empty_batch_is_a_no_op():
    queue = torch.zeros(1, dtype=torch.int32, device=DEV)
    lib.gs_render_fwd_batch(torch.zeros(lib.ctypes.sizeof(lib.GsRasterJob), dtype=torch.uint8, device=DEV), 0, W, H,
                            16, None, queue)
    torch.cuda.synchronize()


def test_project_bwd_accum_adds_exactly_what_project_bwd_writes():
    n = 20000
    P = pu.f32(synth.gaussians_surface(n, 21))
    Pt = torch.from_numpy(pu.pack64(P)).to(DEV)
    cams = [lib.camera(c, tile=16) for c in synth.hemisphere_cameras(2, 4.0, W, H, 60.0)]
    rng = np.random.default_rng(22)
    act_np = np.sort(rng.choice(n, n // 2, replace=False)).astype(np.int32)
    act = torch.from_numpy(act_np).to(DEV)
    na = torch.tensor([len(act_np)], dtype=torch.int32, device=DEV)
    spl, g2d = [], []
    for k, cam in enumerate(cams):
        s = torch.zeros((n, 12), dtype=torch.float32, device=DEV)
        lib.gs_project(Pt, n, 3, cam, s)
        spl.append(s)
        g2d.append(torch.from_numpy(rng.normal(0, 1e-4, (n, 12)).astype(np.float32)).to(DEV))
    Gs = []
    for k in range(2):
        G = torch.full((n, 64), 5.0, device=DEV)
        lib.gs_project_bwd(Pt, n, 3, cams[k], spl[k], act, na, g2d[k].clone(), G)
        Gs.append(G)
    G = torch.full((n, 64), 5.0, device=DEV)
    ax, ar = torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    cnt = torch.zeros(n, dtype=torch.int32, device=DEV)
    ax1, ar1 = torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    cnt1 = torch.zeros(n, dtype=torch.int32, device=DEV)
    lib.gs_project_bwd(Pt, n, 3, cams[1], spl[1], act, na, g2d[1].clone(), torch.zeros_like(G), ax1, ar1, cnt1)
    a, b = g2d[0].clone(), g2d[1].clone()
    lib.gs_project_bwd(Pt, n, 3, cams[0], spl[0], act, na, a, G, ax, ar, cnt)
    ax0, ar0, cnt0 = ax.clone(), ar.clone(), cnt.clone()
    lib.gs_project_bwd_accum(Pt, n, 3, cams[1], spl[1], act, na, b, G, ax, ar, cnt)
    rows = act.long()
    assert torch.equal(G[rows], Gs[0][rows] + Gs[1][rows])
    other = torch.ones(n, dtype=torch.bool, device=DEV)
    other[rows] = False
    assert bool((G[other] == 5.0).all())  # rows of other Gaussians untouched
    assert torch.equal(cnt, cnt0 + cnt1) and torch.equal(ax, ax0 + ax1) and torch.equal(ar, ar0 + ar1)
    visible = spl[1][:, 10].contiguous().view(torch.int32) > 0  # culled Gaussians receive no grad2d at all
    vis_rows = rows[visible[rows]]
    assert not b[vis_rows].any()  # grad2d rows of the visible active Gaussians consumed


def test_devstep_adam_equals_host_step_adam():
    n = 30011
    g = np.random.default_rng(31)
    P0 = torch.from_numpy(g.normal(0, 1, (n, 64)).astype(np.float32)).to(DEV)
    act = torch.from_numpy(np.sort(g.choice(n, 20000, replace=False)).astype(np.int32)).to(DEV)
    na = torch.tensor([20000], dtype=torch.int32, device=DEV)
    lrs = [1e-3, 5e-3, 1e-3, 0.025, 2.5e-3, 1.25e-4]
    lr_dev = torch.tensor(lrs, dtype=torch.float32, device=DEV)
    step_dev = torch.zeros(1, dtype=torch.int64, device=DEV)
    scratch = torch.zeros(2, device=DEV)
    A = [P0.clone(), torch.zeros_like(P0), torch.zeros_like(P0)]
    B = [P0.clone(), torch.zeros_like(P0), torch.zeros_like(P0)]
    for t in range(1, 5):
        G = torch.from_numpy(g.normal(0, 1e-3, (n, 64)).astype(np.float32)).to(DEV)
        lib.gs_adam_masked(A[0], G, A[1], A[2], n, act, na, lrs, 0.9, 0.999, 1e-15, t)
        lib.gs_adam_masked_devstep(B[0], G, B[1], B[2], n, act, na, lr_dev, 0.9, 0.999, 1e-15, step_dev, scratch)
    assert int(step_dev.item()) == 4
    assert torch.allclose(A[1], B[1], rtol=0, atol=0) and torch.allclose(A[2], B[2], rtol=0, atol=0)
    assert torch.allclose(A[0], B[0], rtol=1e-6, atol=1e-7)
    lr_dev[3] = 0.0  # rates are read from device memory when the kernel runs
    before = B[0].clone()
    G = torch.ones((n, 64), device=DEV)
    lib.gs_adam_masked_devstep(B[0], G, B[1], B[2], n, act, na, lr_dev, 0.9, 0.999, 1e-15, step_dev, scratch)
    rows = act.long()
    assert torch.equal(B[0][rows, 10], before[rows, 10])  # opacity column: rate 0
    assert not torch.equal(B[0][rows, 0], before[rows, 0])


# ---- the batch trainer ----
def _tiny_batch(cfg=None, sizes=(1500, 4000, 9000), res=96, views_per_step=2):
    from paper_2504_06716_gb300 import batch
    from paper_2504_06716_gb300.schedule import GStaConfig

    scenes = batch.make_scenes(sizes, res, n_views=18, seed=7)
    return batch.BatchTrainer(scenes, cfg or GStaConfig.tiny(), tile=16, views_per_step=views_per_step)


def _params(bt):
    return [s.model.P[:, :59].clone() for s in bt.scenes]


def _close_training(pa, pb, steps, lrs):
    """Two runs of the same steps whose gradients differ only by the order of
    float atomics: Adam moves a parameter by at most about its rate per step,
    so no entry may differ by more than 2 x steps x rate, and nearly all
    entries must agree far more closely."""
    groups = [(0, 3, 0), (3, 6, 1), (6, 10, 2), (10, 11, 3), (11, 14, 4), (14, 59, 5)]
    for a, b in zip(pa, pb):
        for lo, hi, gi in groups:
            d = (a[:, lo:hi] - b[:, lo:hi]).abs()
            lr = lrs[gi]
            assert float(d.max()) <= 2 * steps * lr * 1.01, (lo, float(d.max()), lr)
            assert float((d > 1e-2 * lr).float().mean()) < 0.01, (lo, float((d > 1e-2 * lr).float().mean()))


def test_graph_replay_trains_like_eager_serial_and_per_job_launches():
    from paper_2504_06716_gb300 import pipeline

    steps = 24
    runs = {}
    for mode in ("graph", "batched", "serial", "per_job"):
        torch.manual_seed(0)
        bt = _tiny_batch()
        launches = [bt.step(mode) for _ in range(steps)]
        assert lib.gs_get_device_error() == 0
        assert all(int(s.step_dev.item()) == steps for s in bt.scenes)
        if mode == "graph":
            assert len(bt.graphs) == bt.n_groups and all(x > 0 for x in launches)
        runs[mode] = (_params(bt), [s.model.frozen.clone() for s in bt.scenes])
    lrs = pipeline.default_lrs(4.4)
    _close_training(runs["graph"][0], runs["batched"][0], steps, lrs)
    _close_training(runs["per_job"][0], runs["batched"][0], steps, lrs)
    _close_training(runs["serial"][0], runs["batched"][0], steps, lrs)


def test_batch_trains_scenes_to_completion_and_they_leave_the_batch():
    bt = _tiny_batch()
    s0 = [s.psnr_of(s.scene.test_views) for s in bt.scenes]
    k = 0
    sizes_seen = set()
    while not bt.finished() and k < 2000:
        bt.step("graph")
        sizes_seen.add(len(bt.active))
        k += 1
    assert bt.finished()
    assert lib.gs_get_device_error() == 0
    s1 = [s.psnr_of(s.scene.test_views) for s in bt.scenes]
    assert all(b > a + 1.0 for a, b in zip(s0, s1)), (s0, s1)
    for s in bt.scenes:
        kinds = {e[1] for e in s.events}
        assert "psnr" in kinds
    assert len(sizes_seen) >= 1


def test_autotuner_picks_a_working_shape():
    from paper_2504_06716_gb300 import batch

    bt = _tiny_batch()
    res = batch.tune(bt, tiles=(8, 16, 32), ppts=(1, 2), batches=(32, 256), reps=1)
    assert res["tile"] in (8, 16, 32) and bt.tile == res["tile"]
    assert set(res["table"]) == {8, 16, 32}
    for _ in range(3):
        bt.step("graph")
    assert lib.gs_get_device_error() == 0
