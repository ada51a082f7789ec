"""veg_bin_sort_static -- binning for callers that cannot allocate device
memory (inside someone else's stream capture, in allocation-free real-time
loops, in plug-ins whose host owns all device memory) -- must produce exactly
what veg_bin_sort produces with a caller workspace.

Several scenes are binned back to back through the same fixed scratch, the
largest first, so stale contents left by one call would show in the next:
a 200,000-record scene (above the 65,536 records below which the binning
sorts every record directly, so the visible-record compaction also runs
through the static array), a three-view scene and the 4096-Gaussian plain
scene, then a capacity overflow whose truncated lists must match too."""
import numpy as np
import pytest
import torch

from paper_2504_13339_gb300 import _lib, scenes as S
from paper_2504_13339_gb300.render import SplatPipeline, lut_tensor

pytestmark = pytest.mark.gpu

STATIC_BYTES = 16 << 20  # size of the library's fixed scratch array


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _scenes():
    big = S.uniform_gaussians(200_000, 35, logscale_mean=-4.2, logscale_std=0.3)
    cams_big = [S.orbit_camera(20.0, 10.0, 3.0, 256, 192)]
    g1, cams1, tf1 = S.plain_scene()
    g2 = S.uniform_gaussians(2000, 31, logscale_mean=-3.0, logscale_std=0.4)
    cams2 = S.orbit_cameras(3, 33, 100, 70)
    return [(big, cams_big, S.bump_tfs(1, 36)), (g2, cams2, S.bump_tfs(3, 34)),
            (g1, cams1, tf1)]


def _workspace_pipeline(g, cams, tfs, capacity):
    p = SplatPipeline(g.n, cams, n_tf=len(tfs), capacity=capacity)
    p.project(_dev(g.mean_v), _dev(g.logscale_w), _dev(g.quat), lut_tensor(tfs))
    p.bin_sort(want_keys=True)
    return p


def _static_bin(p, capacity):
    keys = torch.zeros(max(capacity, 1), dtype=torch.int64, device="cuda")
    vals = torch.full((max(capacity, 1),), -1, dtype=torch.int32, device="cuda")
    ranges = torch.full_like(p.ranges, -7)
    n_inst = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = _lib.veg_bin_sort_static(p.c_cams, p.n, p.geo, p.tiles, p.rect, capacity, keys,
                                      vals, ranges, n_inst)
    torch.cuda.synchronize()
    return status, keys, vals, ranges, int(n_inst.item())


def test_static_scratch_matches_workspace_binning_on_consecutive_calls():
    sizes = []
    for g, cams, tfs in _scenes():
        p = _workspace_pipeline(g, cams, tfs, 800_000)
        st, m = p.status()
        assert st == _lib.VEG_OK and m > 0
        # the exact capacity the instances need, so the request fits the array
        p = _workspace_pipeline(g, cams, tfs, m)
        need = _lib.veg_bin_sort_workspace_size(p.n, p.V, m, p.W, p.H)
        assert need <= STATIC_BYTES
        sizes.append(p.n * p.V)
        status, keys, vals, ranges, n_inst = _static_bin(p, m)
        assert status == _lib.VEG_OK
        assert n_inst == m
        assert torch.equal(vals[:m], p.vals[:m])
        assert torch.equal(keys[:m], p.keys[:m])
        assert torch.equal(ranges, p.ranges)
    assert sizes[0] > 65_536 and sizes == sorted(sizes, reverse=True)


def test_static_scratch_capacity_overflow_keeps_the_same_truncated_lists():
    g, cams, tfs = _scenes()[1]
    p = _workspace_pipeline(g, cams, tfs, 800_000)
    _, m = p.status()
    cap = m // 3
    p = _workspace_pipeline(g, cams, tfs, cap)
    st, m_ws = p.status()
    assert st == _lib.VEG_ERR_CAPACITY and m_ws == m
    status, keys, vals, ranges, n_inst = _static_bin(p, cap)
    assert status == _lib.VEG_OK  # overflow is reported through the count
    assert n_inst == m > cap
    assert torch.equal(vals[:cap], p.vals[:cap])
    assert torch.equal(keys[:cap], p.keys[:cap])
    assert torch.equal(ranges, p.ranges)


def test_static_scratch_rejects_requests_beyond_its_size():
    g, cams, tfs = S.plain_scene()
    big = 4_000_000  # 12 B per instance alone exceeds the 16 MiB array
    p = SplatPipeline(g.n, cams, n_tf=1, capacity=big)  # outputs sized for the request
    status = _lib.veg_bin_sort_static(p.c_cams, g.n, p.geo, p.tiles, p.rect, big, None, p.vals,
                                      p.ranges, None)
    assert status == 5  # VEG_ERR_UNSUPPORTED, nothing launched
