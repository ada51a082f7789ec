"""veg_bin_sort_static -- binning for callers that cannot allocate device
memory (inside someone else's stream capture, in allocation-free real-time
loops, in plug-ins whose host owns all device memory) -- must produce exactly
what veg_bin_sort produces with a caller workspace.  Two different scenes are
binned back to back through the same fixed scratch, larger one first, so
stale contents from the first call would show in the second."""
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


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _scenes():
    g1, cams1, tf1 = S.plain_scene()
    g2 = S.uniform_gaussians(2000, 31, logscale_mean=-3.0, logscale_std=0.4)
    cams2 = S.orbit_cameras(3, 33, 100, 70)
    return [(g1, cams1, tf1), (g2, cams2, S.bump_tfs(3, 34))]


def test_static_scratch_matches_workspace_binning_on_two_calls():
    for g, cams, tfs in _scenes():
        p = SplatPipeline(g.n, cams, n_tf=len(tfs), capacity=60_000)
        p.project(_dev(g.mean_v), _dev(g.logscale_w), _dev(g.quat), lut_tensor(tfs))
        p.bin_sort(want_keys=True)
        st, m = p.status()
        assert st == _lib.VEG_OK and m > 0
        keys = torch.zeros_like(p.keys)
        vals = torch.full_like(p.vals, -1)
        ranges = torch.full_like(p.ranges, -7)
        n_inst = torch.zeros(1, dtype=torch.int64, device="cuda")
        status = _lib.veg_bin_sort_static(p.c_cams, g.n, p.geo, p.tiles, p.rect, p.capacity,
                                          keys, vals, ranges, n_inst)
        assert status == _lib.VEG_OK
        torch.cuda.synchronize()
        assert int(n_inst.item()) == m
        assert torch.equal(vals[:m], p.vals[:m])
        assert torch.equal(keys[:m], p.keys[:m])
        assert torch.equal(ranges, p.ranges)


def test_static_scratch_rejects_requests_beyond_its_size():
    g, cams, tfs = S.plain_scene()
    big = 4_000_000  # 12 B per instance alone exceeds the 16 MiB array
    p = SplatPipeline(g.n, cams, n_tf=1, capacity=big)  # outputs sized for the request
    status = _lib.veg_bin_sort_static(p.c_cams, g.n, p.geo, p.tiles, p.rect, big, None, p.vals,
                                      p.ranges, None)
    assert status == 5  # VEG_ERR_UNSUPPORTED, nothing launched
