"""Pins of the oracle's forward model against closed forms and invariants
(Eq. 3dgs compositing, App. A.1-A.3 projection, App. A.2 SH basis)."""
import math

import numpy as np
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2501_13975_b300 import synth
from tests.oracle_scenes import NOTHRESH, micro_camera


def _one(mean, scale, quat=(1, 0, 0, 0), op=0.6, dc=(1.0, 2.0, 3.0), extra=None):
    m = np.array(mean, np.float32).reshape(3, 1)
    s = np.array(scale, np.float32).reshape(3, 1)
    q = np.array(quat, np.float32).reshape(4, 1)
    q /= np.linalg.norm(q)
    sh = np.array(dc, np.float32).reshape(3, 1, 1)
    sc = synth.Scene(m, q, s, np.array([op], np.float32), sh, 0)
    return sc


def _concat(a, b):
    return synth.Scene(np.concatenate([a.mean, b.mean], 1), np.concatenate([a.quat, b.quat], 1),
                       np.concatenate([a.scale, b.scale], 1), np.concatenate([a.opacity, b.opacity]),
                       np.concatenate([a.sh, b.sh], 2), 0)


def test_sh_basis_orthonormal():
    """B_i Phi_i are orthonormal on the unit sphere: Gauss-Legendre in cos(theta)
    x uniform phi integrates the degree-6 products exactly."""
    x, w = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phis = 2 * np.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for ct, wt in zip(x, w):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            r = (st * math.cos(ph), st * math.sin(ph), ct)
            y = O.sh_basis(r, 3)
            G += wt * (2 * np.pi / nphi) * np.outer(y, y)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_isotropic_splat_integral_exact():
    """One isotropic splat of screen variance s^2 (incl. low-pass) and opacity
    sigma on black: sum over pixels of c = c~ * sigma * 2 pi s^2 (lattice sum of
    a Gaussian with s >= 2 px equals its integral to ~exp(-2 pi^2 s^2))."""
    cam = micro_camera(W=72, H=72, f=60.0)
    z0, s3 = 4.0, 0.2                           # f s3 / z0 = 3 px
    sc = _one((0, 0, z0), (s3, s3, s3), quat=(0.3, 0.5, -0.2, 0.7), op=0.6)
    cfg = dict(NOTHRESH)
    img = O.render(sc, cam, cfg)["image"]
    pr = O.project(sc, cam, cfg)
    s2 = (60.0 * float(np.float32(s3)) / z0) ** 2 + 0.3     # inputs are FP32
    expect = pr["color"][:, 0] * float(np.float32(0.6)) * 2 * np.pi * s2
    assert np.allclose(img.sum(axis=(1, 2)), expect, rtol=1e-9)
    # the principal point: a centre on the optical axis projects to (cx, cy)
    assert np.allclose(pr["pix"][:, 0], [cam.cx, cam.cy], atol=1e-12)
    assert np.allclose(pr["sigma2d"][:, 0], [s2, 0.0, s2], rtol=1e-12, atol=1e-12)


def test_anisotropic_splat_integral():
    """Any PD screen covariance: sum of G over the lattice = 2 pi sqrt(det Sigma)."""
    cam = micro_camera(W=96, H=80, f=50.0)
    sc = _one((0.3, -0.2, 4.0), (0.35, 0.15, 0.2), quat=(0.9, 0.1, 0.3, -0.2), op=0.5)
    cfg = dict(NOTHRESH)
    img = O.render(sc, cam, cfg)["image"]
    pr = O.project(sc, cam, cfg)
    a, b, c = pr["sigma2d"][:, 0]
    expect = pr["color"][:, 0] * float(np.float32(0.5)) * 2 * np.pi * math.sqrt(a * c - b * b)
    assert np.allclose(img.sum(axis=(1, 2)), expect, rtol=1e-9)


def test_truncated_splat_integral():
    """With the alpha >= 1/255 cut the integral over the support ellipse is
    c~ 2 pi s^2 (sigma - 1/255); the lattice sum differs by the lattice-point
    discrepancy of the ellipse boundary (about 1%)."""
    cam = micro_camera(W=72, H=72, f=60.0)
    sc = _one((0, 0, 4.0), (0.2, 0.2, 0.2), op=0.8)
    img = O.render(sc, cam, dict(t_min=0.0))["image"]
    pr = O.project(sc, cam)
    s2 = 9.3
    expect = pr["color"][:, 0] * 2 * np.pi * s2 * (0.8 - 1 / 255)
    assert np.allclose(img.sum(axis=(1, 2)), expect, rtol=2e-2)


def test_two_splat_depth_order_closed_form():
    """Two concentric isotropic splats: front one composited over the back one,
    sum c = c1 s1' + c2 (s2' - sigma1 sigma2 2 pi s1^2 s2^2 / (s1^2 + s2^2)),
    s_i' = sigma_i 2 pi s_i^2. Swapping the depths swaps the roles."""
    cam = micro_camera(W=96, H=96, f=60.0)
    a = _one((0, 0, 3.0), (0.15, 0.15, 0.15), op=0.7, dc=(2.0, 0.0, 0.5))
    b = _one((0, 0, 5.0), (0.4, 0.4, 0.4), op=0.5, dc=(0.0, 2.5, 1.0))
    cfg = dict(NOTHRESH)
    for sc, (front, back) in [(_concat(a, b), (0, 1)), (_concat(b, a), (1, 0))]:
        img = O.render(sc, cam, cfg)["image"]
        pr = O.project(sc, cam, cfg)
        s2 = [pr["sigma2d"][0, i] for i in range(2)]
        sg = [float(v) for v in sc.opacity]
        c = pr["color"]
        f, k = front, back
        cross = sg[f] * sg[k] * 2 * np.pi * s2[f] * s2[k] / (s2[f] + s2[k])
        expect = c[:, f] * sg[f] * 2 * np.pi * s2[f] + c[:, k] * (sg[k] * 2 * np.pi * s2[k] - cross)
        assert np.allclose(img.sum(axis=(1, 2)), expect, rtol=1e-9)


def test_weights_sum_to_one_minus_T():
    """With every c~ = 1 the image equals sum_k alpha_k T_k = 1 - T_final <= 1,
    and T_final >= t_min (compositing stops before T falls below t_min)."""
    sc = synth.tiny_scene(n=400)
    sc.sh[:, 0, :] = 2.0 * math.sqrt(math.pi)        # c~ = 1 with the DC basis 1/(2 sqrt(pi))
    cam = synth.ring_cameras(4, 64)[1]
    r = O.render(sc, cam)
    for ch in range(3):
        assert np.allclose(r["image"][ch], 1.0 - r["tfinal"], atol=1e-12)
    assert r["tfinal"].min() >= 1e-4 and r["image"].max() <= 1.0 + 1e-12
    assert r["ncontrib"].max() > 5


def test_projection_jacobian_sigma_points():
    """Sigma2D - lowpass = J W R S S^T R^T W^T J^T is the linearised pushforward
    of the 3D covariance: compare with the covariance of the projected sigma
    points of a tiny Gaussian (pinhole x/z), relative error O(s^2)."""
    cam = micro_camera(eye=(0.5, 0.2, -0.3), target=(0.1, 0.0, 4.0), W=64, H=48, f=55.0)
    mean = np.array([0.4, -0.25, 3.7])
    quat = np.array([0.8, -0.2, 0.4, 0.3])
    quat /= np.linalg.norm(quat)
    eps = 1e-4
    s = np.array([2.0, 1.0, 0.5]) * eps
    sc = _one(mean, s, quat=quat)
    sc.mean = mean.reshape(3, 1)                       # keep FP64 input
    sc.scale = s.reshape(3, 1)
    sc.quat = quat.reshape(4, 1)
    pr = O.project(sc, cam, dict(lowpass=0.0))
    R = Rotation.from_quat([quat[1], quat[2], quat[3], quat[0]]).as_matrix()
    L = R @ np.diag(s)
    V = np.asarray(cam.viewmat, np.float64)
    pts = []
    for i in range(3):
        for sgn in (1, -1):
            pts.append(mean + sgn * math.sqrt(3) * L[:, i])
    proj = []
    for p in pts:
        t = V[:, :3] @ p + V[:, 3]
        proj.append([cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy])
    proj = np.array(proj)
    mu = proj.mean(0)
    cov = (proj - mu).T @ (proj - mu) / 6.0
    got = np.array([[pr["sigma2d"][0, 0], pr["sigma2d"][1, 0]], [pr["sigma2d"][1, 0], pr["sigma2d"][2, 0]]])
    assert np.abs(got - cov).max() <= 1e-5 * np.abs(cov).max()
    t = V[:, :3] @ mean + V[:, 3]
    assert np.allclose(pr["pix"][:, 0], [cam.fx * t[0] / t[2] + cam.cx, cam.fy * t[1] / t[2] + cam.cy], atol=1e-12)


def test_fov_edge_projects_to_image_edge():
    """A point on the edge of the horizontal field of view lands on the outer
    edge of the pixel grid (x = W - 1/2) with pixel centres at integers."""
    cam = synth.pinhole(128, 96, 60.0, synth.look_at((0, 0, 0), (0, 0, 1)))
    z = 3.0
    x = -z * math.tan(math.radians(30.0))    # camera x axis is world -x for this pose
    sc = _one((x, 0.0, z), (0.01, 0.01, 0.01))
    pr = O.project(sc, cam)
    assert abs(pr["pix"][0, 0] - (128 - 0.5)) < 1e-4


def test_color_uses_view_direction():
    """c~ = sum_i c_i (B_i Phi_i)(r) with r the unit camera->centre direction."""
    sc = synth.tiny_scene(n=5, sh_degree=3, seed=9)
    sc.sh[:, 1:, :] = np.random.default_rng(3).normal(0, 0.5, sc.sh[:, 1:, :].shape)
    cam = synth.ring_cameras(4, 64)[2]
    pr = O.project(sc, cam)
    o = cam.center()
    for k in range(5):
        r = sc.mean[:, k].astype(np.float64) - o
        r /= np.linalg.norm(r)
        y = O.sh_basis(r, 3)
        assert np.allclose(pr["color"][:, k], sc.sh[:, :, k].astype(np.float64) @ y, rtol=1e-12)


def test_depth_order_and_ties():
    """Global order = (FP32 depth key, index); equal keys keep index order."""
    a = _one((0.1, 0, 4.0), (0.2, 0.2, 0.2))
    b = _one((-0.1, 0, 4.0), (0.2, 0.2, 0.2))
    c = _one((0.0, 0.1, 3.0), (0.2, 0.2, 0.2))
    sc = _concat(_concat(a, b), c)
    cam = micro_camera(W=32, H=32)
    assert list(O.order(sc, cam)) == [2, 0, 1]
    pr = O.project(sc, cam)
    assert pr["key"][0] == pr["key"][1]


def test_near_plane_cull():
    sc = _concat(_one((0, 0, 0.19), (0.1, 0.1, 0.1)), _one((0, 0, 0.21), (0.1, 0.1, 0.1)))
    pr = O.project(sc, micro_camera())
    assert list(pr["culled"]) == [True, False]


def test_knn_ring_known_answer():
    """Cameras on a ring around the scene centre: great-circle distance is the
    ring angle times the sphere radius; neighbours sorted by angle."""
    ang = np.radians([0, 10, 30, 60, 100, 150, 210, 280])
    cen = np.stack([5 * np.cos(ang), np.zeros_like(ang), 5 * np.sin(ang)], 1)
    sc = synth.tiny_scene(n=50)
    sphere = O.bounding_sphere(sc)
    cen = cen + sphere[:3]
    nb, dist = O.knn(cen, sphere, 3)
    assert list(nb[0]) == [1, 2, 3]
    assert list(nb[7]) == [6, 0, 1]
    assert abs(dist[0, 1] - sphere[3] * math.radians(10)) < 1e-9


def test_bounding_sphere():
    sc = synth.tiny_scene(n=300)
    s = O.bounding_sphere(sc)
    m = sc.mean.astype(np.float64)
    assert np.allclose(s[:3], 0.5 * (m.min(1) + m.max(1)))
    assert abs(s[3] - np.linalg.norm(m - s[:3, None], axis=0).max()) < 1e-12
