"""The allocation-free freeze update (gs_freeze_update_noalloc).

Some callers cannot allocate device memory at the point where they call
this library -- a host that owns every device buffer and passes in only
inputs and outputs, or a loop that must not call cudaMalloc because an
allocation can synchronise the device. For them the library offers one
entry point whose scratch is a fixed array inside the library. This test
calls it through the C ABI and checks it against gs_freeze_update (which
takes a caller workspace) on two calls in a row; the outputs are integers
and must agree exactly. It lives in a file of its own that is collected
last and sets up everything it needs, so it passes alone or after the rest.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2504_06716_gb300 import lib  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_06716_gb300 import build

    build.build()
    lib.load()


def _inputs(n, seed):
    g = np.random.default_rng(seed)
    acc_x = (g.exponential(3e-5, n) * g.integers(0, 4, n)).astype(np.float32)
    acc_r = (g.exponential(1e-4, n) * g.integers(0, 4, n)).astype(np.float32)
    cnt = g.integers(0, 4, n).astype(np.int32)
    return acc_x, acc_r, cnt


def _state(n, frozen):
    return dict(frozen=torch.from_numpy(frozen.copy()).cuda(),
                act=torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda"),
                na=torch.zeros(1, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("n,modes", [(5000, (0, 0)), (1_300_001, (0, 0)), (70_001, (1, 0)), (70_001, (2, 0)),
                                     (70_001, (0, 1)), (0, (0, 2))])
def test_noalloc_matches_workspace_version_on_two_calls(n, modes):
    """Two calls in a row (update, reset or clear; an empty set too), each
    against gs_freeze_update on the same inputs."""
    frozen0 = (np.random.default_rng(n).uniform(0, 1, n) < 0.1).astype(np.uint8)
    ref, new = _state(n, frozen0), _state(n, frozen0)
    ws = torch.zeros(max(lib.gs_freeze_workspace_bytes(n), 256), dtype=torch.uint8, device="cuda")
    L = lib.load()
    for call, mode in enumerate(modes):
        acc_x, acc_r, cnt = _inputs(n, call + 1)
        a = [torch.from_numpy(x.copy()).cuda() for x in (acc_x, acc_r, cnt)]
        b = [torch.from_numpy(x.copy()).cuda() for x in (acc_x, acc_r, cnt)]
        lib.gs_freeze_update(n, *a, ref["frozen"], 4e-5, 1.1e-4, mode, ref["act"], ref["na"], ws)
        st = L.gs_freeze_update_noalloc(n, b[0].data_ptr(), b[1].data_ptr(), b[2].data_ptr(),
                                        new["frozen"].data_ptr(), 4e-5, 1.1e-4, mode, new["act"].data_ptr(),
                                        new["na"].data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == 0, lib.gs_status_string(st)
        torch.cuda.synchronize()
        k = int(ref["na"].item())
        assert int(new["na"].item()) == k, f"call {call}"
        assert torch.equal(new["frozen"], ref["frozen"]), f"call {call}"
        assert torch.equal(new["act"][:k], ref["act"][:k]), f"call {call}"
        for x in b:
            assert not x.any()
        if mode == 0 and n:
            assert k < n  # the rule froze something, so the comparison is not vacuous
        if mode == 1:
            assert k == n  # a reset unfreezes everything
    assert lib.gs_get_device_error() == 0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = lib.load()
    too_many = 65536 * 1024 + 1
    st = L.gs_freeze_update_noalloc(too_many, None, None, None, None, 1.0, 1.0, 0, None,
                                    ctypes.c_void_p(1), None)
    assert st == 1 and lib.gs_status_string(st) == "invalid argument"
