"""The no-allocation render entry point (gs2_render_noalloc) against the
regular gs2_project + gs2_raster_fwd path, through the C ABI.

It exists for callers that cannot call cudaMalloc (a plugin whose host
application owns all device memory, a real-time loop that must not allocate):
its scratch is a fixed array inside the library.  The array keeps the previous
call's contents, so two calls in a row, on different views, must both match
the regular path.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2501_13975_b300 import synth  # noqa: E402


def test_render_noalloc_matches_regular_path_twice():
    from paper_2501_13975_b300 import gs2
    sc = synth.tiny_scene(n=1000, seed=5, sh_degree=1)
    cams = synth.ring_cameras(4, 128) + [synth.ring_cameras(4, 100, height=75)[1]]
    ds = gs2.DeviceScene.from_host(sc)
    ctx = gs2.Context(sc.n, 128, 128, 1)
    status = torch.full((1,), 77, dtype=torch.int32, device="cuda")
    for cam in (cams[0], cams[4]):          # two calls in a row, different views and sizes
        proj = ctx.project(ds, cam)
        ref_img, ref_rs = ctx.raster_fwd(ds, cam, proj)
        proj2 = ctx.proj_buffer(sc.n)
        img = torch.full_like(ref_img, -1.0)
        rs = ctx.raster_state_buffer(cam.width, cam.height)
        gs2.render_noalloc(ds, cam, proj2, img, rs, status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert float((img - ref_img).abs().max()) <= 1e-5
        tf, last = ctx.raster_state(rs, cam.width, cam.height)
        rtf, rlast = ctx.raster_state(ref_rs, cam.width, cam.height)
        assert float((tf - rtf).abs().max()) <= 1e-5
        assert torch.equal(last, rlast)
        assert float(img.abs().sum()) > 0


def test_render_noalloc_rejects_too_many_tiles():
    from paper_2501_13975_b300 import gs2
    sc = synth.tiny_scene(n=10, seed=5)
    ds = gs2.DeviceScene.from_host(sc)
    cam = synth.ring_cameras(4, 1040)[0]          # 65 x 65 tiles > 4096
    proj = gs2.Context.empty_bytes(gs2._lib.gs2_proj_bytes(sc.n))
    img = torch.empty((3, 1040, 1040), device="cuda")
    rs = gs2.Context.empty_bytes(gs2._lib.gs2_raster_state_bytes(1040, 1040))
    with pytest.raises(gs2.GS2Error, match="ERR_SHAPE"):
        gs2.render_noalloc(ds, cam, proj, img, rs)


def test_render_noalloc_reports_pair_overflow_per_call():
    """More (tile, Gaussian) pairs than GS2_NOALLOC_MAX_PAIRS: the call still
    returns GS2_OK, with GS2_ERR_CAPACITY's bit (1) in the status word, and the
    next call within the limits reports 0 (each call writes its own status).
    1,000 Gaussians with scales near 0.5 seen from 3 units at 1024x1024 list
    about 2.3M pairs against a limit of 524,288."""
    from paper_2501_13975_b300 import gs2
    big = synth.tiny_scene(n=1000, seed=7, log_scale=(-0.7, 0.1))
    small = synth.tiny_scene(n=1000, seed=5, sh_degree=1)
    cam_big = synth.ring_cameras(4, 1024)[0]
    cam_small = synth.ring_cameras(4, 128)[0]
    status = torch.zeros((1,), dtype=torch.int32, device="cuda")
    for sc, cam, want in ((big, cam_big, 1), (small, cam_small, 0), (big, cam_big, 1), (small, cam_small, 0)):
        ds = gs2.DeviceScene.from_host(sc)
        proj = gs2.Context.empty_bytes(gs2._lib.gs2_proj_bytes(sc.n))
        img = torch.empty((3, cam.height, cam.width), device="cuda")
        rs = gs2.Context.empty_bytes(gs2._lib.gs2_raster_state_bytes(cam.width, cam.height))
        gs2.render_noalloc(ds, cam, proj, img, rs, status)   # raises unless GS2_OK
        torch.cuda.synchronize()
        assert int(status.item()) == want, (cam.width, int(status.item()))
        assert bool(torch.isfinite(img).all())
