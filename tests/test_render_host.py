"""Host logic of the differentiable render (no GPU): the library calls are
replaced by recorders, so only the sequencing in Python runs.  A backward
must follow its own forward on a pipeline: a second composite in between
makes it raise instead of differentiating the wrong render."""
import numpy as np
import pytest
import torch


@pytest.fixture
def fake_library(monkeypatch):
    from paper_2504_13339_gb300 import _lib, build
    build.build()  # the workspace-size queries are host functions of the library
    calls = []
    for name in ("veg_project", "veg_bin_sort", "veg_tile_order", "veg_composite_fwd",
                 "veg_composite_bwd"):
        monkeypatch.setattr(_lib, name, lambda *a, _n=name, **k: calls.append(_n))
    monkeypatch.setattr(_lib, "veg_sync_status", lambda *a, **k: (_lib.VEG_OK, 0))
    return calls


def test_backward_needs_its_own_forward(fake_library):
    from paper_2504_13339_gb300 import render as R, scenes as S
    g, cams, tfs = S.plain_scene()
    g = g.subset(np.arange(50))
    p = R.SplatPipeline(g.n, cams, n_tf=1, device="cpu")
    luts = R.lut_tensor(tfs, device="cpu")
    leaf = lambda a: torch.as_tensor(np.ascontiguousarray(a)).requires_grad_()
    mv, ls, q = leaf(g.mean_v), leaf(g.logscale_w), leaf(g.quat)

    out = R.render(mv, ls, q, p, luts)
    assert fake_library == ["veg_project", "veg_bin_sort", "veg_tile_order", "veg_composite_fwd"]
    out.sum().backward()
    assert fake_library[-1] == "veg_composite_bwd"
    assert mv.grad is not None and mv.grad.shape == mv.shape

    first = R.render(mv, ls, q, p, luts)
    second = R.render(mv, ls, q, p, luts)
    n_bwd = fake_library.count("veg_composite_bwd")
    with pytest.raises(RuntimeError, match="composited again"):
        first.sum().backward()
    assert fake_library.count("veg_composite_bwd") == n_bwd  # nothing ran
    second.sum().backward()
    assert fake_library.count("veg_composite_bwd") == n_bwd + 1
