"""The bounded waits of the binning's radix passes on the device: for sorts
of up to 64 chunks each pass is one kernel in which a CTA waits for the
digit counts of the chunks before it.  Sorting seeded keys through veg_radix_lookback_check gives the stable
sort; with the first chunk never taken (the counts its successor waits for
are never published) the wait runs out after its poll limit, the kernel
finishes, veg_sync_status reports VEG_ERR_TIMEOUT, and the GPU keeps
working."""
import numpy as np
import pytest
import torch

from paper_2504_13339_gb300 import _lib, scenes as S
from paper_2504_13339_gb300.render import SplatPipeline, lut_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _check(n, starve, spins):
    ws = torch.empty(_lib.veg_bin_sort_workspace_size(n, 1, 0, 16, 16), dtype=torch.uint8,
                     device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    vals = torch.empty(n, dtype=torch.int32, device="cuda")
    _lib.veg_radix_lookback_check(ws, n, starve, spins, keys, vals)
    st, _ = _lib.veg_sync_status(ws)
    return st, keys.cpu().numpy().view(np.uint32), vals.cpu().numpy().view(np.uint32)


def test_radix_sort_with_bounded_waits_is_the_stable_sort():
    n = 9 * 2048 + 77  # ten chunks, the last ragged
    st, k, v = _check(n, starve=False, spins=1 << 20)
    assert st == _lib.VEG_OK
    i = np.arange(n, dtype=np.uint64)
    ref_keys = ((i * 2654435761) % (1 << 32) >> 4).astype(np.uint32)
    order = np.argsort(ref_keys, kind="stable")
    assert np.array_equal(v, order.astype(np.uint32))
    assert np.array_equal(k, ref_keys[order])


def test_a_wait_that_runs_out_reports_a_timeout_and_the_gpu_keeps_working():
    st, _, _ = _check(9 * 2048 + 77, starve=True, spins=1 << 12)
    assert st == _lib.VEG_ERR_TIMEOUT
    # the context is intact: a full binning and render afterwards match as before
    g, cams, tfs = S.plain_scene()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    p = SplatPipeline(g.n, cams, n_tf=1)
    out = p.render(t(g.mean_v), t(g.logscale_w), t(g.quat), lut_tensor(tfs)).clone()
    assert p.status()[0] == _lib.VEG_OK
    q = SplatPipeline(g.n, cams, n_tf=1)
    assert torch.equal(q.render(t(g.mean_v), t(g.logscale_w), t(g.quat), lut_tensor(tfs)), out)


def test_a_sort_beyond_the_look_back_limit_is_refused():
    n = 64 * 2048 + 1
    ws = torch.empty(_lib.veg_bin_sort_workspace_size(n, 1, 0, 16, 16), dtype=torch.uint8,
                     device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(_lib.VegError):
        _lib.veg_radix_lookback_check(ws, n, False, 1 << 20, keys, keys)
