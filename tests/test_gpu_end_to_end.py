"""End-to-end parity of the autograd form (all stages on the GPU) with the
oracle: images, gradients of every primitive parameter, central finite
differences, invariants, edge cases and the full-size headline workload on
sampled pixels."""
import numpy as np
import pytest
import torch

from paper_2606_11529_gb300 import binding as B
from paper_2606_11529_gb300 import render as R
from paper_2606_11529_gb300 import scenes

from gpu_util import BAND_E2E, GRAD_TOL, check_band, dev, rel_err

pytestmark = pytest.mark.gpu

NAMES = ["mu", "scale", "quat", "opacity", "sh"]


def _params(sc):
    return [t.clone().requires_grad_(True) for t in R.scene_to_device(sc)]


def test_small_case_image_and_gradients(oracle):
    """10k Gaussians, 256x256, 16x16 tiles: image and all five gradients vs the FP64 tiled oracle."""
    sc, cam, cfg = scenes.small_case()
    ref = oracle.pipeline_tiled(sc, cam, cfg, band=BAND_E2E)
    P = _params(sc)
    img = R.render(*P, cam, cfg)
    got = img.detach().cpu().numpy()
    # band: gate decisions within the float32 uncertainty of the kernels' own projection (0.44% of
    # this image's pixels; their error is bounded by the jump of the flagged decisions)
    check_band(got, ref, max_frac=1e-2, what="small case")
    w = np.random.default_rng(0).normal(size=got.shape) * ~ref["gband"][None]
    (img * dev(w)).sum().backward()
    d_rec = oracle.render_bwd_tiles(ref["proj"]["rec"], ref["vals"], ref["ranges"], cam, cfg, w)
    g = oracle.project_bwd(*sc.arrays(), cam, cfg, d_rec)
    for name, p in zip(NAMES, P):
        assert rel_err(p.grad.cpu().numpy(), g[name]) < GRAD_TOL, name


@pytest.mark.parametrize("deg,tile", [(3, 16), (1, 8)])
def test_sh_scene_with_view_and_background(oracle, deg, tile):
    sc = scenes.uniform_scene(6000, seed=3, sh_degree=deg)
    cam = scenes.pinhole(224, 160, 224.0, scenes.yaw_view(-6.0, (0.1, 0.05, -0.2)))
    cfg = scenes.RenderConfig(tile_w=tile, tile_h=tile, sh_degree=deg, bg=(0.25, 0.5, 0.75))
    ref = oracle.pipeline_tiled(sc, cam, cfg, band=BAND_E2E)
    P = _params(sc)
    img = R.render(*P, cam, cfg)
    got = img.detach().cpu().numpy()
    check_band(got, ref, max_frac=1e-2, what=f"SH {deg}, {tile}x{tile} tiles, rotated view")
    w = np.random.default_rng(1).normal(size=got.shape) * ~ref["gband"][None]
    (img * dev(w)).sum().backward()
    d_rec = oracle.render_bwd_tiles(ref["proj"]["rec"], ref["vals"], ref["ranges"], cam, cfg, w)
    g = oracle.project_bwd(*sc.arrays(), cam, cfg, d_rec)
    for name, p in zip(NAMES, P):
        assert rel_err(p.grad.cpu().numpy(), g[name]) < GRAD_TOL, name


def test_gradients_match_central_differences(oracle):
    """GPU gradients vs central finite differences of the FP64 forward on a tiny scene."""
    rng = np.random.default_rng(11)
    n, deg = 6, 3
    mu = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(2.5, 4.0, n)], 1)
    s = np.exp(rng.normal(-1.6, 0.3, (n, 3)))
    q = rng.normal(size=(n, 4))
    o = 1 / (1 + np.exp(-rng.normal(0.5, 0.8, n)))
    sh = rng.normal(0, 0.3, (n, 16, 3))
    sh[:, 0, :] = rng.uniform(0.5, 1.5, (n, 3))
    Pn = [a.astype(np.float32).astype(np.float64) for a in (mu, s, q, o, sh)]
    cam = scenes.pinhole(32, 32, 32.0)
    cfg = scenes.RenderConfig(sh_degree=deg, bg=(0.1, 0.2, 0.3))
    w = rng.normal(size=(3, 32, 32))
    P = [dev(a).requires_grad_(True) for a in Pn]
    img = R.render(*P, cam, cfg)
    (img * dev(w)).sum().backward()
    for a, name in enumerate(NAMES):
        fd = np.zeros_like(Pn[a])
        it = np.nditer(Pn[a], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            x0 = Pn[a][idx]
            h = 1e-6 * max(abs(x0), 1e-2)
            Pp = [p.copy() for p in Pn]
            Pm = [p.copy() for p in Pn]
            Pp[a][idx] = x0 + h
            Pm[a][idx] = x0 - h
            lp, sp = oracle.loss_brute(Pp, cam, cfg, w)
            lm, sm = oracle.loss_brute(Pm, cam, cfg, w)
            fd[idx] = (lp - lm) / (2 * h) if sp == sm else np.nan
        m = ~np.isnan(fd)
        assert m.mean() > 0.97
        assert rel_err(P[a].grad.cpu().numpy()[m], fd[m]) < GRAD_TOL, name


def test_input_permutation_gives_identical_image():
    sc, cam, cfg = scenes.small_case()
    a = R.forward_frame(*R.scene_to_device(sc), cam, cfg).image
    perm = np.random.default_rng(0).permutation(sc.n)
    b = R.forward_frame(*R.scene_to_device(sc.subset(perm)), cam, cfg).image
    assert torch.equal(a, b)
    c = R.forward_frame(*R.scene_to_device(sc), cam, cfg).image
    assert torch.equal(a, c)  # the forward is deterministic


def test_tile_size_invariance():
    sc, cam, _ = scenes.small_case()
    im = {t: R.forward_frame(*R.scene_to_device(sc), cam, scenes.RenderConfig(tile_w=t, tile_h=t)).image
          for t in (8, 16)}
    d = (im[8] - im[16]).abs()
    assert (d > 1e-6).float().mean().item() < 1e-3 and d.max().item() < 5e-3


def test_telescoping_white_on_gpu():
    sc, cam, cfg = scenes.small_case()
    sc.sh[:, 0, :] = 0.5 * np.sqrt(4 * np.pi)  # colour exactly 1
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    np.testing.assert_allclose(fr.image.cpu().numpy(), np.broadcast_to(1 - fr.t_final.cpu().numpy(), (3, 256, 256)),
                               atol=2e-6)


def test_empty_and_all_invisible():
    cam = scenes.pinhole(100, 60, 100.0)
    cfg = scenes.RenderConfig(bg=(0.25, 0.5, 0.75))
    empty = scenes.uniform_scene(0, seed=0)
    fr = R.forward_frame(*R.scene_to_device(empty), cam, cfg)
    assert fr.n_isect == 0
    np.testing.assert_allclose(fr.image.cpu().numpy(), np.array([0.25, 0.5, 0.75])[:, None, None] * np.ones((3, 60, 100)))
    sc = scenes.uniform_scene(500, seed=1)
    sc.mu[:, 2] = -3.0
    P = _params(sc)
    img = R.render(*P, cam, cfg)
    img.sum().backward()
    assert torch.all(img == torch.tensor([0.25, 0.5, 0.75], device="cuda")[:, None, None])
    for p in P:
        assert torch.all(p.grad == 0)


def test_one_huge_gaussian_covers_every_tile(oracle):
    sc = scenes.uniform_scene(3, seed=2)
    sc.mu[:] = [[0.0, 0.0, 2.0], [0.1, 0.0, 3.0], [-0.1, 0.05, 4.0]]
    sc.scale[:] = [[2.0, 1.5, 1.0], [0.05, 0.05, 0.05], [0.3, 0.1, 0.2]]
    cam = scenes.pinhole(128, 96, 128.0)
    cfg = scenes.RenderConfig()
    ref = oracle.pipeline_tiled(sc, cam, cfg, band=BAND_E2E)
    fr = R.forward_frame(*R.scene_to_device(sc), cam, cfg)
    assert fr.n_isect >= 8 * 6
    check_band(fr.image.cpu().numpy(), ref, max_frac=1e-2, what="huge Gaussian")


def test_capacity_retry_inside_the_path():
    sc, cam, cfg = scenes.small_case()
    ws = R.Workspace()
    a = R.forward_frame(*R.scene_to_device(sc), cam, cfg, ws)
    assert ws.last_isect == a.n_isect
    ws.last_isect = 0  # force a too-small first guess
    b = R.forward_frame(*R.scene_to_device(sc), cam, cfg, ws)
    assert torch.equal(a.image, b.image) and a.n_isect == b.n_isect


def test_headline_workload_sampled_pixels_and_gradients(oracle):
    """1M SH-3 Gaussians, 1920x1080, 16x16 tiles (the benchmarked launch configuration):
    sampled pixels vs the brute-force oracle, and gradients from a sparse loss on those pixels."""
    sc, cam, cfg = scenes.headline_case()
    P = _params(sc)
    img = R.render(*P, cam, cfg)
    torch.cuda.synchronize()
    pr = oracle.project_scene(sc, cam, cfg)
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(0, 1920, 384), rng.integers(0, 1080, 384)], 1)
    # brute force over all primitives in the order of the float32 depth keys (the kernels' order)
    ref = oracle.render_pixels(pr["rec"], pix, cfg, band=BAND_E2E, key=pr["key"], unc=pr["unc"])
    got = img.detach().cpu().numpy()[:, pix[:, 1], pix[:, 0]].T
    ok = check_band(got, ref, max_frac=1e-2, what="1M / 1080p sampled pixels")
    ok &= ~ref["gband"]
    assert (ref["t_final"] < 0.5).mean() > 0.2  # sampled pixels are not mostly empty
    # sparse loss on the unambiguous sampled pixels
    use = pix[ok][:128]
    w = np.zeros((3, 1080, 1920))
    w[:, use[:, 1], use[:, 0]] = rng.normal(size=(3, len(use)))
    (img * dev(w)).sum().backward()
    d_rec = oracle.render_bwd_brute(pr["rec"], cam, cfg, w, key=pr["key"])
    g = oracle.project_bwd(*sc.arrays(), cam, cfg, d_rec)
    for name, p in zip(NAMES, P):
        assert rel_err(p.grad.cpu().numpy(), g[name]) < GRAD_TOL, name


def test_deferred_colour_equals_one_pass():
    # projection without colours while the SH coefficients are still being copied, then
    # xpr_project_color: the same image bit for bit, and the same gradients
    sc = scenes.clustered_scene(30_000, seed=11, n_centers=40, width=320, height=180, focal=320.0, sh_degree=3)
    cam = scenes.pinhole(320, 180, 320.0, scenes.yaw_view(3.0, (0.02, 0.0, 0.05)))
    cfg = scenes.RenderConfig(sh_degree=3, bg=(0.2, 0.1, 0.0))
    P = [t.requires_grad_(True) for t in R.scene_to_device(sc)]
    ref = R.forward_frame(*[p.detach() for p in P], cam, cfg).image
    host_sh = torch.from_numpy(sc.sh).pin_memory()
    dev_sh = torch.zeros_like(P[4].detach())
    up = R.Uploader()
    ev = up.start([dev_sh], [host_sh])
    fr = R.forward_frame(*[p.detach() for p in P[:4]], dev_sh, cam, cfg, sh_events=ev)
    assert torch.equal(fr.image, ref)
    w = torch.from_numpy(np.random.default_rng(4).normal(size=tuple(ref.shape)).astype(np.float32)).cuda()
    (R.render(*P, cam, cfg) * w).sum().backward()
    g_ref = [p.grad.clone() for p in P]
    for p in P:
        p.grad = None
    ws = R.Workspace()
    with torch.no_grad():
        P[4].zero_()
    ws.sh_events = up.start([P[4].detach()], [host_sh])
    (R.render(*P, cam, cfg, ws) * w).sum().backward()
    for a, b in zip(g_ref, P):
        assert rel_err(b.grad.cpu().numpy(), a.cpu().numpy()) < 1e-5


def test_projection_from_pinned_host_equals_resident():
    # inputs still in pinned host memory: the projection reads the geometry over the host link and
    # writes its device copy in the same pass, then the SH coefficients are copied under the binning
    # and sort: the frame equals the one from resident inputs bit for bit, the device copy equals the
    # host data, and the gradients through the autograd function are those of resident inputs
    sc = scenes.clustered_scene(30_001, seed=12, n_centers=40, width=320, height=180, focal=320.0, sh_degree=3)
    cam = scenes.pinhole(320, 180, 320.0, scenes.yaw_view(3.0, (0.02, 0.0, 0.05)))
    cfg = scenes.RenderConfig(sh_degree=3, bg=(0.2, 0.1, 0.0))
    P = [t.requires_grad_(True) for t in R.scene_to_device(sc)]
    ref = R.forward_frame(*[p.detach() for p in P], cam, cfg, R.Workspace(rows_counts=True))
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in sc.arrays()]
    up = R.Uploader()
    dst = [torch.zeros_like(p.detach()) for p in P]
    rec, bbox, tc, cnt = B.xpr_project_host(host[:4], dst[:4] + [None], cam, cfg, with_isect_count=True)
    for a, b in zip((ref.bbox, ref.tile_count, ref.isect_count), (bbox, tc, cnt)):
        assert torch.equal(a, b)
    for d, h in zip(dst[:4], host[:4]):
        assert torch.equal(d.cpu(), h)
    dst = [torch.zeros_like(p.detach()) for p in P]
    fr = R.forward_frame(*dst, cam, cfg, R.Workspace(rows_counts=True), host_inputs=(host, up.stream))
    for name in ("rec", "bbox", "tile_count", "isect_count", "vals_sorted", "ranges", "image", "t_final", "n_contrib"):
        assert torch.equal(getattr(ref, name), getattr(fr, name)), name
    w = torch.from_numpy(np.random.default_rng(5).normal(size=tuple(ref.image.shape)).astype(np.float32)).cuda()
    (R.render(*P, cam, cfg) * w).sum().backward()
    g_ref = [p.grad.clone() for p in P]
    for p in P:
        p.grad = None
    with torch.no_grad():
        for p in P:
            p.zero_()
    ws = R.Workspace()
    ws.host_inputs = (host, up.stream)
    (R.render(*P, cam, cfg, ws) * w).sum().backward()
    for a, b in zip(g_ref, P):
        assert rel_err(b.grad.cpu().numpy(), a.cpu().numpy()) < 1e-5
    # pageable host memory is refused before any launch
    pageable = [torch.from_numpy(np.ascontiguousarray(a)) for a in sc.arrays()[:4]]
    with pytest.raises(B.XprError):
        B.xpr_project_host(pageable, dst[:4] + [None], cam, cfg)
