"""The volume raymarcher on the GPU vs the oracle (ground-truth renderer of
the paper's training images, Sec. 4.2 / 5.1).

Bars: prepared gradients within float32 rounding; images within 1e-4
max-abs per channel on unflagged pixels (the oracle flags pixels whose
sample count or stop decision sits at a float32 boundary), at a small size
in full and at the training size (800 x 800, 256^3 volume, 10 maps) on
sampled pixels.
"""
import numpy as np
import pytest
import torch

from oracle import veg_raymarch_oracle as RM
from paper_2504_13339_gb300 import _lib, scenes as S
from paper_2504_13339_gb300.render import lut_tensor
from paper_2504_13339_gb300.train import opacity_guided_luts

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
MAT = (0.3, 0.6, 0.25, 12.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


def prepared(vol):
    v = dev(vol)
    v4 = torch.empty(vol.shape + (4,), device="cuda")
    _lib.veg_volume_prepare(v, v4)
    return v4


def march(cams, v4, luts, step, material=None, bg=(0.0, 0.0, 0.0), view_tf=None):
    lt = lut_tensor(luts)
    n_out = 1 if view_tf is not None else lt.shape[0]
    out = torch.empty(len(cams), n_out, cams[0].height, cams[0].width, 4, device="cuda")
    vt = None if view_tf is None else torch.as_tensor(np.asarray(view_tf, np.int32),
                                                      device="cuda")
    _lib.veg_raymarch(_lib.cameras(cams), v4, _lib.tf_desc(lt, vt), step, out, material, bg)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_prepared_gradients_match_oracle():
    vol = S.field_volume(S.blob_field(5, 100), 21)
    v4 = prepared(vol).cpu().numpy()
    ref = RM.vertex_gradients(vol)
    assert np.array_equal(v4[..., 0], vol)
    scale = np.abs(ref).max()
    assert np.abs(v4[..., 1:] - ref).max() <= 2e-6 * scale


@pytest.mark.parametrize("material,bg", [(None, (0.0, 0.0, 0.0)), (MAT, (0.1, 0.2, 0.3))])
def test_raymarch_matches_oracle(material, bg):
    vol = S.field_volume(S.blob_field(5, 101), 17)
    cams = S.orbit_cameras(2, 102, 40, 28)  # ragged: 3 x 2 tiles
    luts = S.bump_tfs(3, 103)
    h = 2.0 / 16
    got = march(cams, prepared(vol), luts, h / 2, material, bg)
    flagged = 0
    for v, cam in enumerate(cams):
        ref, flag = RM.render(cam, vol.astype(np.float64), luts.astype(np.float64), h / 2,
                              material, bg)
        err = np.abs(got[v] - ref)
        ok = ~flag
        assert np.all(err[ok] <= IMG_TOL), float(err[ok].max())
        flagged += int(flag.sum())
    assert flagged <= 0.01 * got[..., 0].size


def test_one_table_per_view_equals_the_slice():
    vol = S.field_volume(S.blob_field(4, 104), 17)
    cams = S.orbit_cameras(3, 105, 32, 32)
    luts = S.bump_tfs(3, 106)
    v4 = prepared(vol)
    full = march(cams, v4, luts, 0.06, MAT)
    one = march(cams, v4, luts, 0.06, MAT, view_tf=[2, 0, 1])
    for v, t in enumerate([2, 0, 1]):
        assert np.array_equal(one[v, 0], full[v, t])


def test_training_size_on_sampled_pixels():
    """256^3 volume, 800 x 800, the 10 opacity-guided maps, shaded: 24
    random pixels of one view against the oracle ray by ray."""
    bf = S.blob_field(8, 107)
    vol = S.field_volume(bf, 256)
    cam = S.grid_orbit_cameras(16, 10, 800, 800)[37]
    luts = opacity_guided_luts(10, S.colour_ramp(108))
    step = (2.0 / 255) / 2
    got = march([cam], prepared(vol), luts, step, MAT)
    rng = np.random.default_rng(109)
    vol64 = vol.astype(np.float64)
    checked = 0
    for _ in range(24):
        i, j = int(rng.integers(150, 650)), int(rng.integers(150, 650))
        ref, flag = RM.march_pixel(cam, vol64, luts.astype(np.float64), i, j, step, MAT)
        for t in range(10):
            if flag[t]:
                continue
            assert np.all(np.abs(got[0, t, j, i] - ref[t]) <= IMG_TOL), (i, j, t)
            checked += 1
    assert checked >= 200


def test_instrumented_run_is_identical_and_counts_samples():
    vol = S.field_volume(S.blob_field(4, 110), 17)
    cams = S.orbit_cameras(2, 111, 40, 28)
    luts = S.bump_tfs(3, 112)
    v4 = prepared(vol)
    plain = march(cams, v4, luts, 0.06, MAT)
    lt = lut_tensor(luts)
    out = torch.empty(len(cams), 3, 28, 40, 4, device="cuda")
    st = torch.zeros(2, dtype=torch.int64, device="cuda")
    _lib.veg_raymarch(_lib.cameras(cams), v4, _lib.tf_desc(lt), 0.06, out, MAT, stats=st)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), plain)
    samples, tables = (int(x) for x in st.cpu().numpy())
    # every sample of a ray evaluates at most the three tables of its group
    assert 0 < samples <= tables <= 3 * samples
    # no ray is longer than the box diagonal
    assert samples <= 2 * 40 * 28 * (2 * 3 ** 0.5 / 0.06 + 1)


def cell_masks_numpy(vol, luts, cell):
    """The macrocell table masks by their definition, in float32 like the
    kernel: vertex range of each macrocell, widened by 1e-6, the table
    entries it interpolates between plus one on each side."""
    R, L = vol.shape[0], luts.shape[1]
    c = -(-(R - 1) // cell)
    m = np.zeros((c, c, c), np.uint32)
    f32 = np.float32
    for z in range(c):
        for y in range(c):
            for x in range(c):
                blk = vol[z * cell:min(z * cell + cell, R - 1) + 1,
                          y * cell:min(y * cell + cell, R - 1) + 1,
                          x * cell:min(x * cell + cell, R - 1) + 1]
                if np.isnan(blk).any() or luts.shape[0] > 32:
                    m[z, y, x] = 0xffffffff
                    continue
                lo = min(max(f32(blk.min()) - f32(1e-6), f32(0)), f32(1)) * f32(L - 1)
                hi = min(max(f32(blk.max()) + f32(1e-6), f32(0)), f32(1)) * f32(L - 1)
                k0, k1 = max(int(np.floor(lo)) - 1, 0), min(int(np.floor(hi)) + 2, L - 1)
                for t in range(luts.shape[0]):
                    if (luts[t, k0:k1 + 1, 3] > 0).any():
                        m[z, y, x] |= np.uint32(1 << t)
    return m.ravel()


@pytest.mark.parametrize("cell", [2, 4])
def test_cell_masks_follow_their_definition(cell):
    vol = S.field_volume(S.blob_field(4, 113), 19)  # 18 vertex cells: ragged at cell 4
    luts = opacity_guided_luts(10, S.colour_ramp(114))
    v4 = prepared(vol)
    n = _lib.veg_raymarch_cells_count(19, cell)
    assert n == (-(-18 // cell)) ** 3
    mask = torch.zeros(n, dtype=torch.int32, device="cuda")
    _lib.veg_raymarch_cells(v4, _lib.tf_desc(lut_tensor(luts)), cell, mask)
    got = mask.cpu().numpy().view(np.uint32)
    ref = cell_masks_numpy(vol, luts, cell)
    assert np.array_equal(got, ref)
    # many macrocells hold only values where map 0 (opaque at 0) has opacity
    assert (got == 1).sum() > n // 3 and len(np.unique(got)) > 4


def masked_and_plain(vol, cams, luts, step, material, view_tf=None, cell=4):
    v4 = prepared(vol)
    lt = lut_tensor(luts)
    vt = None if view_tf is None else torch.as_tensor(np.asarray(view_tf, np.int32),
                                                      device="cuda")
    tf = _lib.tf_desc(lt, vt)
    n_out = 1 if view_tf is not None else lt.shape[0]
    shape = (len(cams), n_out, cams[0].height, cams[0].width, 4)
    plain, masked = torch.empty(shape, device="cuda"), torch.empty(shape, device="cuda")
    st0 = torch.zeros(2, dtype=torch.int64, device="cuda")
    st1 = torch.zeros(3, dtype=torch.int64, device="cuda")
    c_cams = _lib.cameras(cams)
    _lib.veg_raymarch(c_cams, v4, tf, step, plain, material, stats=st0)
    mask = torch.empty(_lib.veg_raymarch_cells_count(vol.shape[0], cell), dtype=torch.int32,
                       device="cuda")
    _lib.veg_raymarch_cells(v4, _lib.tf_desc(lt), cell, mask)
    _lib.veg_raymarch_masked(c_cams, v4, tf, step, masked, mask, cell, material, stats=st1)
    torch.cuda.synchronize()
    return plain.cpu().numpy(), masked.cpu().numpy(), st0.cpu().numpy(), st1.cpu().numpy()


def test_masked_raymarch_is_bit_identical_and_skips():
    """Skipping macrocells whose live tables have no opacity changes no
    image bit; taken + skipped samples equal the plain run's samples."""
    vol = S.field_volume(S.blob_field(6, 115), 33)
    cams = S.orbit_cameras(2, 116, 40, 28)
    luts = opacity_guided_luts(10, S.colour_ramp(117))
    plain, masked, st0, st1 = masked_and_plain(vol, cams, luts, 2.0 / 32 / 2, MAT)
    assert np.array_equal(plain, masked)
    assert st1[0] + st1[2] == st0[0] and st1[2] > 0 and st1[1] <= st0[1]
    one_p, one_m, _, _ = masked_and_plain(vol, cams, luts, 0.04, None, view_tf=[9, 3])
    assert np.array_equal(one_p, one_m)


def test_masked_raymarch_at_training_size():
    """256^3 volume, 800 x 800, the 10 maps, shaded: masked images equal the
    plain ones for two views, and most samples are skipped."""
    vol = S.field_volume(S.blob_field(8, 118), 256)
    cams = S.grid_orbit_cameras(16, 10, 800, 800)[40:42]
    luts = opacity_guided_luts(10, S.colour_ramp(119))
    plain, masked, st0, st1 = masked_and_plain(vol, cams, luts, (2.0 / 255) / 2, MAT, cell=8)
    assert np.array_equal(plain, masked)
    assert st1[0] + st1[2] == st0[0] and st1[2] > st1[0]
