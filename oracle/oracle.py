"""ctypes front end of the FP64 CPU oracle (liboracle.so, built from gs2_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline legs of bench.py. It never imports the CUDA package, and the
CUDA package never imports it.

Scenes and cameras are duck-typed: any object with the attributes of
synth.Scene / synth.Camera works (mean, quat, scale, opacity, sh, sh_degree;
width, height, fx, fy, cx, cy, viewmat).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SRC_PATH = os.path.join(HERE, "gs2_oracle.c")

POS, ROT, SCALE, OPACITY, COLOR = 0, 1, 2, 3, 4
GROUPS = (POS, ROT, SCALE, OPACITY, COLOR)

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_fp = C.POINTER(C.c_float)


class OrcScene(C.Structure):
    _fields_ = [("n", C.c_int), ("sh_degree", C.c_int), ("mean", _dp), ("quat", _dp), ("scale", _dp),
                ("opacity", _dp), ("sh", _dp)]


class OrcCamera(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("viewmat", C.c_double * 12),
                ("clip_x", C.c_double), ("clip_y", C.c_double)]


class OrcConfig(C.Structure):
    _fields_ = [("lambda_ssim", C.c_double), ("alpha_min", C.c_double), ("alpha_max", C.c_double),
                ("t_min", C.c_double), ("lowpass", C.c_double), ("near_z", C.c_double),
                ("barrier_alpha", C.c_double), ("frac_to_boundary", C.c_double),
                ("damping_mu0", C.c_double), ("damping_tries", C.c_int), ("scale_min", C.c_double),
                ("ssim_c1", C.c_double), ("ssim_c2", C.c_double), ("ssim_sigma", C.c_double),
                ("ssim_radius", C.c_int), ("knn_k", C.c_int), ("downsample", C.c_int),
                ("scale_trust", C.c_double), ("trust_pos", C.c_double), ("trust_rot", C.c_double),
                ("trust_color", C.c_double), ("gauss_newton", C.c_int), ("group_order", C.c_int * 5),
                ("group_jacobi", C.c_int), ("gd_lr", C.c_double * 5)]


def default_config(**kw) -> dict:
    """The oracle's defaults (the readings of the paper's unstated constants)."""
    cfg = dict(lambda_ssim=0.2, alpha_min=1.0 / 255.0, alpha_max=0.99, t_min=1e-4, lowpass=0.3,
               near_z=0.2, barrier_alpha=1e-6, frac_to_boundary=0.99, damping_mu0=1.0,
               damping_tries=6, scale_min=1e-7, ssim_c1=0.01 ** 2, ssim_c2=0.03 ** 2, ssim_sigma=1.5,
               ssim_radius=5, knn_k=3, downsample=2, scale_trust=1.05,
               trust_pos=0.05, trust_rot=0.05, trust_color=0.05,
               gauss_newton=0, group_order=(0, 1, 2, 3, 4), group_jacobi=0, gd_lr=(0.0, 0.0, 0.0, 0.0, 0.0),
               learned_trust=1.0)
    cfg.update(kw)
    return cfg


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < max(
            os.path.getmtime(SRC_PATH), os.path.getmtime(os.path.join(HERE, "jet.h"))):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", LIB_PATH, SRC_PATH, "-lm"])
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB_PATH)
        L.orc_loss.restype = C.c_double
        L.orc_solve.restype = C.c_int
        _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


class _SceneHandle:
    """Holds FP64 copies of a scene so the C struct's pointers stay valid."""

    def __init__(self, scene):
        self.n = int(scene.mean.shape[1])
        self.sh_degree = int(scene.sh_degree)
        self.mean = np.array(scene.mean, dtype=np.float64, order="C", copy=True)
        self.quat = np.array(scene.quat, dtype=np.float64, order="C", copy=True)
        self.scale = np.array(scene.scale, dtype=np.float64, order="C", copy=True)
        self.opacity = np.array(scene.opacity, dtype=np.float64, order="C", copy=True)
        self.sh = np.array(scene.sh, dtype=np.float64, order="C", copy=True)
        self.c = OrcScene(self.n, self.sh_degree, _d(self.mean), _d(self.quat), _d(self.scale),
                          _d(self.opacity), _d(self.sh))

    def arrays(self):
        return dict(mean=self.mean, quat=self.quat, scale=self.scale, opacity=self.opacity, sh=self.sh)


def scene_handle(scene) -> _SceneHandle:
    return scene if isinstance(scene, _SceneHandle) else _SceneHandle(scene)


def cam_struct(cam) -> OrcCamera:
    c = OrcCamera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    vm = np.asarray(cam.viewmat, np.float64).reshape(-1)
    for i in range(12):
        c.viewmat[i] = vm[i]
    c.clip_x = float(getattr(cam, "clip_x", 0.0))
    c.clip_y = float(getattr(cam, "clip_y", 0.0))
    return c


def cfg_struct(cfg: dict | None) -> OrcConfig:
    d = default_config() if cfg is None else default_config(**cfg)
    c = OrcConfig()
    for k, _ in OrcConfig._fields_:
        if k == "group_order":
            order = [int(x) for x in d[k]]
            if sorted(order) != [0, 1, 2, 3, 4]:
                raise ValueError(f"group_order must be a permutation of 0..4: {order}")
            c.group_order = (C.c_int * 5)(*order)
        elif k == "gd_lr":
            c.gd_lr = (C.c_double * 5)(*[float(x) for x in d[k]])
        else:
            setattr(c, k, d[k])
    return c


def sh_count(degree: int) -> int:
    return (degree + 1) ** 2


def group_dims(group: int, S: int) -> int:
    return {POS: 3, ROT: 1, SCALE: 3, OPACITY: 1, COLOR: S}[group]


# ----------------------------------------------------------------------------- API

def sh_basis(r, degree: int) -> np.ndarray:
    out = np.zeros(sh_count(degree), np.float64)
    lib().orc_sh_basis(C.c_double(r[0]), C.c_double(r[1]), C.c_double(r[2]), C.c_int(degree), _d(out))
    return out


def project(scene, cam, cfg=None):
    sh = scene_handle(scene)
    n = sh.n
    out = np.zeros((15, n), np.float64)
    key = np.zeros(n, np.float32)
    lib().orc_project(C.byref(sh.c), C.byref(cam_struct(cam)), C.byref(cfg_struct(cfg)), _d(out),
                      key.ctypes.data_as(_fp))
    return dict(pix=out[0:2], sigma2d=out[2:5], conic=out[5:8], opacity=out[8], color=out[9:12],
                tz=out[12], culled=out[13].astype(bool), key=key)


def render(scene, cam, cfg=None):
    sh = scene_handle(scene)
    W, H = int(cam.width), int(cam.height)
    img = np.zeros((3, H, W), np.float64)
    tf = np.zeros((H, W), np.float64)
    nc = np.zeros((H, W), np.int32)
    mg = np.zeros((H, W), np.float64)
    lib().orc_render(C.byref(sh.c), C.byref(cam_struct(cam)), C.byref(cfg_struct(cfg)), _d(img), _d(tf),
                     nc.ctypes.data_as(_ip), _d(mg))
    return dict(image=img, tfinal=tf, ncontrib=nc, margin=mg)


def loss(image, target, cfg=None, derivs=True):
    image = np.ascontiguousarray(image, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    _, H, W = image.shape
    e = np.zeros_like(image) if derivs else None
    h = np.zeros_like(image) if derivs else None
    parts = np.zeros(2, np.float64)
    L = lib().orc_loss(_d(image), _d(target), C.c_int(W), C.c_int(H), C.byref(cfg_struct(cfg)),
                       _d(e) if derivs else None, _d(h) if derivs else None, _d(parts))
    return dict(loss=L, l2=parts[0], lssim=parts[1], e=e, h=h)


def ssim_map(image, target, cfg=None):
    """Per-pixel SSIM [3][H][W] and its window moments [3][5][H][W]
    (mu_x, mu_y, E x^2, E y^2, E xy), as L_S averages them."""
    image = np.ascontiguousarray(image, np.float64)
    target = np.ascontiguousarray(target, np.float64)
    _, H, W = image.shape
    out = np.zeros_like(image)
    mom = np.zeros((3, 5, H, W))
    lib().orc_ssim_map(_d(image), _d(target), C.c_int(W), C.c_int(H), C.byref(cfg_struct(cfg)), _d(out), _d(mom))
    return out, mom


def block_shapes(group: int, n: int, S: int):
    if group == COLOR:
        return (3, S, n), (3, S * (S + 1) // 2, n)
    D = group_dims(group, S)
    return (D, n), (D * (D + 1) // 2, n)


def accum(group, scene, view, primary, e, h, cfg=None, out=None):
    """Adds the group's block contributions of one view. Returns dict g, H, gabs, Habs, npix."""
    sh = scene_handle(scene)
    S = sh_count(sh.sh_degree)
    gs, hs = block_shapes(group, sh.n, S)
    if out is None:
        out = dict(g=np.zeros(gs), H=np.zeros(hs), gabs=np.zeros(gs), Habs=np.zeros(hs),
                   npix=np.zeros(sh.n, np.int32))
    e = np.ascontiguousarray(e, np.float64)
    h = np.ascontiguousarray(h, np.float64)
    lib().orc_accum(C.c_int(group), C.byref(sh.c), C.byref(cam_struct(view)), C.byref(cam_struct(primary)),
                    C.byref(cfg_struct(cfg)), _d(e), _d(h), _d(out["g"]), _d(out["H"]), _d(out["gabs"]),
                    _d(out["Habs"]), out["npix"].ctypes.data_as(_ip))
    return out


def solve(group, scene, primary, g, H, cfg=None):
    sh = scene_handle(scene)
    n, S = sh.n, sh_count(sh.sh_degree)
    if group == COLOR:
        step = np.zeros((3, S, n))
        status = np.zeros((3, n), np.int32)
        info = np.zeros((3, 3, n))
        cond = np.zeros((3, n))
    else:
        D = {POS: 3, ROT: 1, SCALE: 3, OPACITY: 1}[group]
        step = np.zeros((D, n))
        status = np.zeros(n, np.int32)
        info = np.zeros((3, n))
        cond = np.zeros(n)
    g = np.ascontiguousarray(g, np.float64)
    H = np.ascontiguousarray(H, np.float64)
    nfail = lib().orc_solve(C.c_int(group), C.byref(sh.c), C.byref(cam_struct(primary)), C.byref(cfg_struct(cfg)),
                            _d(g), _d(H), _d(step), status.ctypes.data_as(_ip), _d(info), _d(cond))
    return dict(step=step, status=status, info=info, cond=cond, nfail=nfail)


def reduced_basis(group, scene, primary, cfg=None):
    """[n][3][2] basis of the reduced position / scaling solve, its status [n]
    and, for scaling, how close the reduction is to degenerate [n]."""
    sh = scene_handle(scene)
    B = np.zeros((sh.n, 3, 2))
    st = np.zeros(sh.n, np.int32)
    gap = np.zeros(sh.n)
    r = lib().orc_reduced_basis(C.c_int(group), C.byref(sh.c), C.byref(cam_struct(primary)),
                                C.byref(cfg_struct(cfg)), _d(B), st.ctypes.data_as(_ip), _d(gap))
    if r != 0:
        raise ValueError("reduced_basis: position or scaling only")
    return B, st, gap


def apply(group, scene, primary, step, cfg=None):
    """Returns a new FP64 scene handle with the step applied."""
    src = scene_handle(scene)
    dst = _SceneHandle(src)
    step = np.ascontiguousarray(step, np.float64)
    lib().orc_apply(C.c_int(group), C.byref(dst.c), C.byref(cam_struct(primary)), C.byref(cfg_struct(cfg)),
                    _d(step))
    return dst


def bounding_sphere(scene) -> np.ndarray:
    sh = scene_handle(scene)
    out = np.zeros(4)
    lib().orc_bounding_sphere(C.byref(sh.c), _d(out))
    return out


def knn(centres, sphere, K):
    centres = np.ascontiguousarray(centres, np.float64)
    m = centres.shape[0]
    out = np.zeros((m, K), np.int32)
    dist = np.zeros((m, m))
    lib().orc_knn(C.c_int(m), _d(centres), _d(np.ascontiguousarray(sphere, np.float64)), C.c_int(K),
                  out.ctypes.data_as(_ip), _d(dist))
    return out, dist


class _Cam:
    def __init__(self, c: OrcCamera):
        self.width, self.height = c.width, c.height
        self.fx, self.fy, self.cx, self.cy = c.fx, c.fy, c.cx, c.cy
        self.viewmat = np.array(list(c.viewmat)).reshape(3, 4)
        self.clip_x, self.clip_y = c.clip_x, c.clip_y


def downsample_camera(cam, f):
    out = OrcCamera()
    lib().orc_downsample_camera(C.byref(cam_struct(cam)), C.c_int(f), C.byref(out))
    return _Cam(out)


def downsample_image(img, f):
    img = np.ascontiguousarray(img, np.float64)
    _, H, W = img.shape
    out = np.zeros((3, H // f, W // f))
    lib().orc_downsample_image(_d(img), C.c_int(W), C.c_int(H), C.c_int(f), _d(out))
    return out


def sweep(scene, cams, targets, knn_table, t, cfg=None):
    """One full sweep for primary t. Returns (new scene handle, losses[5], nfail)."""
    dst = _SceneHandle(scene_handle(scene))
    arr = (OrcCamera * len(cams))(*[cam_struct(c) for c in cams])
    tg = np.ascontiguousarray(targets, np.float64)
    kt = np.ascontiguousarray(knn_table, np.int32)
    losses = np.zeros(5)
    nfail = C.c_int(0)
    lib().orc_sweep(C.byref(dst.c), arr, _d(tg), C.c_int(len(cams)), kt.ctypes.data_as(_ip), C.c_int(t),
                    C.byref(cfg_struct(cfg)), _d(losses), C.byref(nfail))
    return dst, losses, nfail.value


def tile_touch(scene, cam, tile, cfg=None):
    sh = scene_handle(scene)
    W, H = int(cam.width), int(cam.height)
    tx, ty = (W + tile - 1) // tile, (H + tile - 1) // tile
    touch = np.zeros((ty * tx, sh.n), np.uint8)
    rect = np.zeros((4, sh.n))
    lib().orc_tile_touch(C.byref(sh.c), C.byref(cam_struct(cam)), C.byref(cfg_struct(cfg)), C.c_int(tile),
                         touch.ctypes.data_as(C.POINTER(C.c_ubyte)), _d(rect))
    return touch, rect


def dec32(scene, cam, cfg=None):
    """FP32 decision records [18][n] (the layout of the library's projection dump;
    rows 15, 16 hold the tile rectangle's words as bit patterns)."""
    sh = scene_handle(scene)
    out = np.zeros((18, sh.n), np.float32)
    lib().orc_dec32(C.byref(sh.c), C.byref(cam_struct(cam)), C.byref(cfg_struct(cfg)), out.ctypes.data_as(_fp))
    return out


def tile_lists(scene, cam, cfg=None):
    """Tile lists of 16x16 tiles by plain loops: (ranges [ntiles][2], ids)."""
    sh = scene_handle(scene)
    W, H = int(cam.width), int(cam.height)
    nt = ((W + 15) // 16) * ((H + 15) // 16)
    ranges = np.zeros((nt, 2), np.uint32)
    L = lib()
    L.orc_tile_lists.restype = C.c_longlong
    up = C.POINTER(C.c_uint)
    cap = 1 << 16
    while True:
        ids = np.zeros(cap, np.uint32)
        m = L.orc_tile_lists(C.byref(sh.c), C.byref(cam_struct(cam)), C.byref(cfg_struct(cfg)),
                             ranges.ctypes.data_as(up), ids.ctypes.data_as(up), C.c_longlong(cap))
        if m <= cap:
            return ranges, ids[:m]
        cap = int(m)


def order(scene, cam, cfg=None):
    sh = scene_handle(scene)
    out = np.zeros(sh.n, np.int32)
    m = lib().orc_order(C.byref(sh.c), C.byref(cam_struct(cam)), C.byref(cfg_struct(cfg)), out.ctypes.data_as(_ip))
    return out[:m]


def to_fp32_scene(handle, like):
    """FP32 copy of an oracle scene (used to start the next group from the same FP32 state)."""
    s = like.copy()
    s.mean = handle.mean.astype(np.float32)
    s.quat = handle.quat.astype(np.float32)
    s.scale = handle.scale.astype(np.float32)
    s.opacity = handle.opacity.astype(np.float32)
    s.sh = handle.sh.astype(np.float32)
    return s
