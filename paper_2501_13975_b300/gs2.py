"""ctypes binding of libgs2.so (include/gs2.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels; PyTorch only
provides device memory and the stream. Importing this module raises if the
compiled library is missing (build it with ``python -m
paper_2501_13975_b300.build``); there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs2.so")

POS, ROT, SCALE, OPACITY, COLOR = 0, 1, 2, 3, 4
GROUPS = (POS, ROT, SCALE, OPACITY, COLOR)
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_SHAPE", 3: "ERR_CUDA", 4: "ERR_OOM", 5: "ERR_NONFINITE",
          6: "ERR_TIMEOUT", 7: "ERR_UNSUPPORTED", 8: "ERR_CAPACITY"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libgs2.so not found at {LIB_PATH}; build it with `python -m paper_2501_13975_b300.build`")

_lib = C.CDLL(LIB_PATH)

_vp = C.c_void_p


class Scene_(C.Structure):
    _fields_ = [("n", C.c_int32), ("sh_degree", C.c_int32), ("mean", _vp), ("quat", _vp), ("scale", _vp),
                ("opacity", _vp), ("sh", _vp)]


class Camera_(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("viewmat", C.c_float * 12),
                ("clip_x", C.c_float), ("clip_y", C.c_float)]


class Config_(C.Structure):
    _fields_ = [("lambda_ssim", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("t_min", C.c_float), ("lowpass", C.c_float), ("near_z", C.c_float),
                ("barrier_alpha", C.c_float), ("frac_to_boundary", C.c_float), ("damping_mu0", C.c_float),
                ("damping_tries", C.c_int32), ("scale_min", C.c_float), ("scale_trust", C.c_float),
                ("trust_pos", C.c_float), ("trust_rot", C.c_float), ("trust_color", C.c_float),
                ("ssim_c1", C.c_float), ("ssim_c2", C.c_float), ("ssim_sigma", C.c_float),
                ("ssim_radius", C.c_int32), ("knn_k", C.c_int32), ("downsample", C.c_int32),
                ("precision", C.c_int32), ("gauss_newton", C.c_int32), ("group_order", C.c_int32 * 5),
                ("group_jacobi", C.c_int32), ("gd_lr", C.c_float * 5), ("deterministic", C.c_int32),
                ("learned_trust", C.c_float)]


class Tuning_(C.Structure):
    _fields_ = [("sort_blocks", C.c_int32), ("sort_rows", C.c_int32), ("view_lanes", C.c_int32),
                ("accum_px", C.c_int32), ("accum_split", C.c_int32)]


def _tuning_dict(t) -> dict:
    return dict(sort_blocks=t.sort_blocks, sort_rows=t.sort_rows, view_lanes=t.view_lanes, accum_px=t.accum_px,
                accum_split=t.accum_split)


class BatchScene_(C.Structure):
    _fields_ = [("max_gaussians", C.c_int64), ("max_width", C.c_int32), ("max_height", C.c_int32),
                ("max_sh_degree", C.c_int32), ("max_pairs", C.c_int64)]


_sigs = {
    "gs2_config_default": (None, [C.POINTER(Config_)]),
    "gs2_create": (C.c_int, [C.POINTER(_vp), C.POINTER(Config_), C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                             C.c_int64]),
    "gs2_destroy": (C.c_int, [_vp]),
    "gs2_last_error": (C.c_char_p, [_vp]),
    "gs2_set_config": (C.c_int, [_vp, C.POINTER(Config_)]),
    "gs2_check": (C.c_int, [_vp, _vp]),
    "gs2_proj_bytes": (C.c_size_t, [C.c_int64]),
    "gs2_raster_state_bytes": (C.c_size_t, [C.c_int32, C.c_int32]),
    "gs2_blocks_bytes": (C.c_size_t, [C.c_int, C.c_int64, C.c_int32, C.c_int32]),
    "gs2_step_bytes": (C.c_size_t, [C.c_int, C.c_int64, C.c_int32]),
    "gs2_project": (C.c_int, [_vp, C.POINTER(Scene_), C.POINTER(Camera_), _vp, _vp]),
    "gs2_raster_fwd": (C.c_int, [_vp, C.POINTER(Scene_), C.POINTER(Camera_), _vp, _vp, _vp, _vp]),
    "gs2_loss_derivs": (C.c_int, [_vp, _vp, _vp, C.c_int32, C.c_int32, _vp, _vp, _vp, _vp]),
    "gs2_accum_newton_blocks": (C.c_int, [_vp, C.c_int, C.POINTER(Scene_), C.POINTER(Camera_), C.POINTER(Camera_),
                                          _vp, _vp, _vp, _vp, C.c_int32, _vp, _vp, _vp]),
    "gs2_solve_step": (C.c_int, [_vp, C.c_int, _vp, C.c_int32, C.POINTER(Scene_), C.POINTER(Camera_), _vp, _vp,
                                 _vp]),
    "gs2_apply_step": (C.c_int, [_vp, C.c_int, _vp, C.POINTER(Scene_), C.POINTER(Camera_), _vp]),
    "gs2_downsample": (C.c_int, [_vp, _vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp]),
    "gs2_camera_downsample": (None, [C.POINTER(Camera_), C.c_int32, C.POINTER(Camera_)]),
    "gs2_bounding_sphere": (C.c_int, [_vp, C.POINTER(Scene_), _vp, _vp]),
    "gs2_camera_knn": (C.c_int, [_vp, C.c_int32, _vp, C.c_int32, _vp]),
    "gs2_sweep": (C.c_int, [_vp, C.POINTER(Scene_), C.POINTER(Camera_), C.c_int32, C.POINTER(_vp), _vp,
                            C.c_int32, _vp, _vp, _vp]),
    "gs2_sweep_logged": (C.c_int, [_vp, C.POINTER(Scene_), C.POINTER(Camera_), C.c_int32, C.POINTER(_vp), _vp,
                                   C.c_int32, _vp, _vp, _vp, _vp, _vp]),
    "gs2_set_step_model": (C.c_int, [_vp, _vp]),
    "gs2_set_damping_model": (C.c_int, [_vp, _vp]),
    "gs2_step_records": (C.c_int, [_vp, C.c_int, _vp, C.c_int32, C.POINTER(Scene_), _vp, _vp, _vp]),
    "gs2_step_labels": (C.c_int, [_vp, C.c_int, _vp, C.c_int32, C.POINTER(Scene_), _vp, _vp, _vp]),
    "gs2_mlp_forward": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.c_int64, _vp, _vp]),
    "gs2_mlp_grad": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.c_int64, _vp, _vp, _vp, _vp]),
    "gs2_records_chunk_scale": (C.c_int, [_vp, C.c_int64, C.c_int64, _vp, _vp]),
    "gs2_mlp_adam": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_float, C.c_float, C.c_float,
                               C.c_float, _vp]),
    "gs2_get_tuning": (C.c_int, [_vp, C.POINTER(Tuning_)]),
    "gs2_set_tuning": (C.c_int, [_vp, C.POINTER(Tuning_)]),
    "gs2_autotune": (C.c_int, [_vp, C.POINTER(Scene_), C.POINTER(Camera_), C.c_int32, C.POINTER(_vp), _vp,
                               C.c_int32, C.c_int32, C.POINTER(Tuning_), C.POINTER(C.c_float), _vp]),
    "gs2_batch_create": (C.c_int, [C.POINTER(_vp), C.POINTER(Config_), C.c_int32, C.POINTER(BatchScene_)]),
    "gs2_batch_destroy": (C.c_int, [_vp]),
    "gs2_batch_ctx": (_vp, [_vp, C.c_int32]),
    "gs2_batch_last_error": (C.c_char_p, [_vp]),
    "gs2_batch_stats": (C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "gs2_batch_sweep": (C.c_int, [_vp, C.POINTER(Scene_), C.POINTER(C.POINTER(Camera_)), C.POINTER(C.c_int32),
                                  C.POINTER(C.POINTER(_vp)), C.POINTER(C.POINTER(C.c_int32)), C.POINTER(C.c_int32),
                                  _vp, _vp, C.c_int32, _vp]),
    "gs2_launch_count": (C.c_uint64, []),
    "gs2_profile": (C.c_int, [_vp, C.c_int32]),
    "gs2_profile_read": (C.c_int, [_vp, _vp, _vp, _vp]),
    "gs2_profile_read_stages": (C.c_int, [_vp, _vp, _vp]),
    "gs2_fp64_resolves": (C.c_int, [_vp, C.POINTER(C.c_uint64), C.c_int32]),
    "gs2_render_noalloc": (C.c_int, [C.POINTER(Config_), C.POINTER(Scene_), C.POINTER(Camera_), _vp, _vp, _vp,
                                     _vp, _vp]),
    "gs2_debug_tiles": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.POINTER(C.c_int64), _vp]),
    "gs2_debug_keys": (C.c_int, [_vp, C.c_int64, _vp, _vp]),
    "gs2_debug_lookback_timeout": (C.c_int, [_vp, C.c_int32, C.c_uint32, _vp]),
    "gs2_debug_proj": (C.c_int, [_vp, C.c_int64, _vp, _vp]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_sigs)

# learned step scale (include/gs2.h)
MLP_NFEAT, MLP_HIDDEN, MLP_NPARAM, MLP_GRID, REC_ROWS = 8, 64, 4801, 148, 11
DEBUG_PROJ_ROWS = 18   # gs2_debug_proj rows (include/gs2.h)


class GS2Error(RuntimeError):
    pass


def default_config(**kw) -> dict:
    c = Config_()
    _lib.gs2_config_default(C.byref(c))
    d = {k: getattr(c, k) for k, _ in Config_._fields_}
    d["group_order"] = [int(x) for x in c.group_order]
    d["gd_lr"] = [float(x) for x in c.gd_lr]
    for k, v in kw.items():
        if k not in d:
            raise KeyError(k)
        d[k] = [int(x) for x in v] if k == "group_order" else [float(x) for x in v] if k == "gd_lr" else v
    return d


def _config_struct(cfg: dict | None) -> Config_:
    d = default_config(**(cfg or {}))
    c = Config_()
    for k, _ in Config_._fields_:
        if k == "group_order":
            c.group_order = (C.c_int32 * 5)(*[int(x) for x in d[k]])
        elif k == "gd_lr":
            c.gd_lr = (C.c_float * 5)(*[float(x) for x in d[k]])
        else:
            setattr(c, k, d[k])
    return c


def camera_struct(cam) -> Camera_:
    c = Camera_()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    vm = np.asarray(cam.viewmat, np.float32).reshape(-1)
    for i in range(12):
        c.viewmat[i] = float(vm[i])
    c.clip_x = float(getattr(cam, "clip_x", 0.0))
    c.clip_y = float(getattr(cam, "clip_y", 0.0))
    return c


def camera_downsample(cam, f: int) -> Camera_:
    out = Camera_()
    _lib.gs2_camera_downsample(C.byref(camera_struct(cam)), int(f), C.byref(out))
    return out


@dataclasses.dataclass
class DeviceScene:
    """Scene parameters as CUDA tensors in the library's planar layout."""
    mean: torch.Tensor      # (3, n)
    quat: torch.Tensor      # (4, n)
    scale: torch.Tensor     # (3, n)
    opacity: torch.Tensor   # (n,)
    sh: torch.Tensor        # (3, S, n)
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.mean.shape[1])

    @staticmethod
    def from_host(scene, device="cuda") -> "DeviceScene":
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device)
        return DeviceScene(t(scene.mean), t(scene.quat), t(scene.scale), t(scene.opacity), t(scene.sh),
                           int(scene.sh_degree))

    def to_host(self):
        from . import synth
        return synth.Scene(self.mean.cpu().numpy(), self.quat.cpu().numpy(), self.scale.cpu().numpy(),
                           self.opacity.cpu().numpy(), self.sh.cpu().numpy(), self.sh_degree)

    def clone(self) -> "DeviceScene":
        return DeviceScene(self.mean.clone(), self.quat.clone(), self.scale.clone(), self.opacity.clone(),
                           self.sh.clone(), self.sh_degree)

    def struct(self) -> Scene_:
        for t in (self.mean, self.quat, self.scale, self.opacity, self.sh):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        return Scene_(self.n, self.sh_degree, self.mean.data_ptr(), self.quat.data_ptr(), self.scale.data_ptr(),
                      self.opacity.data_ptr(), self.sh.data_ptr())


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous()
    return t.data_ptr()


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def sh_count(degree: int) -> int:
    return (degree + 1) ** 2


class Context:
    """Owns a gs2_ctx (library scratch) on the current CUDA device."""

    def __init__(self, max_gaussians: int, max_width: int, max_height: int, max_sh_degree: int = 3,
                 max_pairs: int = 0, config: dict | None = None):
        self.config = default_config(**(config or {}))
        self._cfg = _config_struct(self.config)
        h = _vp()
        st = _lib.gs2_create(C.byref(h), C.byref(self._cfg), int(max_gaussians), int(max_width), int(max_height),
                             int(max_sh_degree), int(max_pairs))
        if st != 0:
            raise GS2Error(f"gs2_create failed: {STATUS.get(st, st)}")
        self.h = h
        self.max_sh_degree = max_sh_degree

    def close(self):
        if getattr(self, "h", None):
            _lib.gs2_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ok(self, st, what):
        if st != 0:
            msg = _lib.gs2_last_error(self.h).decode() if self.h else ""
            raise GS2Error(f"{what}: {STATUS.get(st, st)} {msg}")

    def set_config(self, **kw):
        self.config = default_config(**{**self.config, **kw})
        self._cfg = _config_struct(self.config)
        self._ok(_lib.gs2_set_config(self.h, C.byref(self._cfg)), "gs2_set_config")

    def check(self, stream=None):
        st = _lib.gs2_check(self.h, _stream(stream))
        self._ok(st, "device status")

    # ---------------------------------------------------------------- buffers
    @staticmethod
    def empty_bytes(nbytes: int, device="cuda"):
        return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device)

    def proj_buffer(self, n):
        return self.empty_bytes(_lib.gs2_proj_bytes(int(n)))

    def raster_state_buffer(self, w, h):
        return self.empty_bytes(_lib.gs2_raster_state_bytes(int(w), int(h)))

    def blocks_buffer(self, group, n, sh_degree, n_views):
        nb = _lib.gs2_blocks_bytes(int(group), int(n), int(sh_degree), int(n_views))
        return torch.zeros(nb // 4, dtype=torch.float32, device="cuda")

    def step_buffer(self, group, n, sh_degree):
        nb = _lib.gs2_step_bytes(int(group), int(n), int(sh_degree))
        return torch.zeros(max(nb // 4, 1), dtype=torch.float32, device="cuda")

    # ---------------------------------------------------------------- calls
    def project(self, scene: DeviceScene, cam, proj=None, stream=None):
        proj = self.proj_buffer(scene.n) if proj is None else proj
        s = scene.struct()
        self._ok(_lib.gs2_project(self.h, C.byref(s), C.byref(camera_struct(cam)), _ptr(proj), _stream(stream)),
                 "gs2_project")
        return proj

    def raster_fwd(self, scene: DeviceScene, cam, proj, image=None, rstate=None, stream=None):
        W, H = int(cam.width), int(cam.height)
        image = torch.empty((3, H, W), dtype=torch.float32, device="cuda") if image is None else image
        rstate = self.raster_state_buffer(W, H) if rstate is None else rstate
        s = scene.struct()
        self._ok(_lib.gs2_raster_fwd(self.h, C.byref(s), C.byref(camera_struct(cam)), _ptr(proj), _ptr(image),
                                     _ptr(rstate), _stream(stream)), "gs2_raster_fwd")
        return image, rstate

    def raster_state(self, rstate, w, h):
        """(tfinal (H,W) float32, last (H,W) int32) views of a raster-state buffer."""
        P = w * h
        a = ((4 * P + 255) // 256) * 256
        tf = rstate[: 4 * P].view(torch.float32).view(h, w)
        last = rstate[a: a + 4 * P].view(torch.int32).view(h, w)
        return tf, last

    def loss_derivs(self, image, target, loss=None, stream=None):
        _, H, W = image.shape
        e = torch.empty_like(image)
        h = torch.empty_like(image)
        self._ok(_lib.gs2_loss_derivs(self.h, _ptr(image), _ptr(target), W, H, _ptr(e), _ptr(h), _ptr(loss),
                                      _stream(stream)), "gs2_loss_derivs")
        return e, h

    def accum(self, group, scene: DeviceScene, view, primary, proj, rstate, image, target, view_slot, blocks,
              loss=None, stream=None):
        s = scene.struct()
        self._ok(_lib.gs2_accum_newton_blocks(self.h, int(group), C.byref(s), C.byref(camera_struct(view)),
                                              C.byref(camera_struct(primary)), _ptr(proj), _ptr(rstate),
                                              _ptr(image), _ptr(target), int(view_slot), _ptr(blocks), _ptr(loss),
                                              _stream(stream)), "gs2_accum_newton_blocks")

    def solve(self, group, blocks, n_views, scene: DeviceScene, primary, step=None, n_failed=None, stream=None):
        step = self.step_buffer(group, scene.n, scene.sh_degree) if step is None else step
        s = scene.struct()
        self._ok(_lib.gs2_solve_step(self.h, int(group), _ptr(blocks), int(n_views), C.byref(s),
                                     C.byref(camera_struct(primary)), _ptr(step), _ptr(n_failed), _stream(stream)),
                 "gs2_solve_step")
        return step

    def apply(self, group, step, scene: DeviceScene, primary, stream=None):
        s = scene.struct()
        self._ok(_lib.gs2_apply_step(self.h, int(group), _ptr(step), C.byref(s), C.byref(camera_struct(primary)),
                                     _stream(stream)), "gs2_apply_step")

    def downsample(self, img, f, stream=None):
        _, H, W = img.shape
        out = torch.empty((3, H // f, W // f), dtype=torch.float32, device="cuda")
        self._ok(_lib.gs2_downsample(self.h, _ptr(img), W, H, int(f), _ptr(out), _stream(stream)), "gs2_downsample")
        return out

    def bounding_sphere(self, scene: DeviceScene, stream=None):
        out = torch.empty(4, dtype=torch.float32, device="cuda")
        s = scene.struct()
        self._ok(_lib.gs2_bounding_sphere(self.h, C.byref(s), _ptr(out), _stream(stream)), "gs2_bounding_sphere")
        return out

    def sweep(self, scene: DeviceScene, cams, targets, knn, t, losses=None, n_failed=None, stream=None):
        arr = (Camera_ * len(cams))(*[camera_struct(c) for c in cams])
        tp = (_vp * len(targets))(*[_ptr(x) for x in targets])
        kt = np.ascontiguousarray(knn, np.int32)
        s = scene.struct()
        self._ok(_lib.gs2_sweep(self.h, C.byref(s), arr, len(cams), tp, kt.ctypes.data_as(_vp), int(t),
                                _ptr(losses), _ptr(n_failed), _stream(stream)), "gs2_sweep")

    def sweep_logged(self, scene: DeviceScene, cams, targets, knn, t, records=None, losses=None, n_failed=None,
                     stream=None, records_damping=None):
        """Plain sweep that logs the records of every group: float [5][REC_ROWS][n]
        (and, with records_damping, the damping network's records of the same shape)."""
        if records is None:
            records = torch.empty((5, REC_ROWS, scene.n), dtype=torch.float32, device="cuda")
        arr = (Camera_ * len(cams))(*[camera_struct(c) for c in cams])
        tp = (_vp * len(targets))(*[_ptr(x) for x in targets])
        kt = np.ascontiguousarray(knn, np.int32)
        s = scene.struct()
        self._ok(_lib.gs2_sweep_logged(self.h, C.byref(s), arr, len(cams), tp, kt.ctypes.data_as(_vp), int(t),
                                       _ptr(records), _ptr(records_damping), _ptr(losses), _ptr(n_failed),
                                       _stream(stream)),
                 "gs2_sweep_logged")
        return records

    def set_damping_model(self, w_bf16):
        """Install (a device int16/uint16 tensor of MLP_NPARAM BF16 words, kept
        alive by this context) or remove (None) the damping network."""
        self._damping_model = w_bf16
        self._ok(_lib.gs2_set_damping_model(self.h, _ptr(w_bf16)), "gs2_set_damping_model")

    def set_step_model(self, w_bf16):
        """Install (a device int16/uint16 tensor of MLP_NPARAM BF16 words, kept
        alive by this context) or remove (None) the step-scale network."""
        self._step_model = w_bf16
        self._ok(_lib.gs2_set_step_model(self.h, _ptr(w_bf16)), "gs2_set_step_model")

    def step_records(self, group, blocks, n_views, scene: DeviceScene, step, records=None, stream=None):
        if records is None:
            records = torch.empty((REC_ROWS, scene.n), dtype=torch.float32, device="cuda")
        s = scene.struct()
        self._ok(_lib.gs2_step_records(self.h, int(group), _ptr(blocks), int(n_views), C.byref(s), _ptr(step),
                                       _ptr(records), _stream(stream)), "gs2_step_records")
        return records

    def step_labels(self, group, blocks_after, n_views, scene: DeviceScene, step, records, stream=None):
        s = scene.struct()
        self._ok(_lib.gs2_step_labels(self.h, int(group), _ptr(blocks_after), int(n_views), C.byref(s), _ptr(step),
                                      _ptr(records), _stream(stream)), "gs2_step_labels")
        return records

    def tuning(self) -> dict:
        t = Tuning_()
        self._ok(_lib.gs2_get_tuning(self.h, C.byref(t)), "gs2_get_tuning")
        return _tuning_dict(t)

    def set_tuning(self, sort_blocks: int | None = None, sort_rows: int | None = None, view_lanes: int | None = None,
                   accum_px: int | None = None, accum_split: int | None = None):
        cur = self.tuning()
        t = Tuning_(int(cur["sort_blocks"] if sort_blocks is None else sort_blocks),
                    int(cur["sort_rows"] if sort_rows is None else sort_rows),
                    int(cur["view_lanes"] if view_lanes is None else view_lanes),
                    int(cur["accum_px"] if accum_px is None else accum_px),
                    int(cur["accum_split"] if accum_split is None else accum_split))
        self._ok(_lib.gs2_set_tuning(self.h, C.byref(t)), "gs2_set_tuning")

    def autotune(self, scene: DeviceScene, cams, targets, knn, t, reps=2, stream=None):
        """Times candidate tunings on a copy of the scene; keeps and returns the fastest."""
        arr = (Camera_ * len(cams))(*[camera_struct(c) for c in cams])
        tp = (_vp * len(targets))(*[_ptr(x) for x in targets])
        kt = np.ascontiguousarray(knn, np.int32)
        s = scene.struct()
        best = Tuning_()
        ms = C.c_float(0.0)
        self._ok(_lib.gs2_autotune(self.h, C.byref(s), arr, len(cams), tp, kt.ctypes.data_as(_vp), int(t),
                                   int(reps), C.byref(best), C.byref(ms), _stream(stream)), "gs2_autotune")
        return dict(_tuning_dict(best), ms=float(ms.value))

    def profile(self, enable: bool):
        self._ok(_lib.gs2_profile(self.h, 1 if enable else 0), "gs2_profile")

    def profile_read(self):
        ms = np.zeros(5, np.float64)
        cnt = np.zeros(5, np.int64)
        stats = np.zeros((5, 6), np.uint64)
        self._ok(_lib.gs2_profile_read(self.h, ms.ctypes.data_as(_vp), cnt.ctypes.data_as(_vp),
                                       stats.ctypes.data_as(_vp)), "gs2_profile_read")
        sms = np.zeros(3, np.float64)
        scnt = np.zeros(3, np.int64)
        self._ok(_lib.gs2_profile_read_stages(self.h, sms.ctypes.data_as(_vp), scnt.ctypes.data_as(_vp)),
                 "gs2_profile_read_stages")
        return dict(accum_ms=ms, accum_launches=cnt, pairs=stats[:, 0], visible=stats[:, 1],
                    binnings=stats[:, 2], pixels=stats[:, 3], evaluations=stats[:, 4], listed=stats[:, 5],
                    stage_ms=dict(binning=sms[0], compositing=sms[1], loss=sms[2]),
                    stage_count=dict(binning=int(scnt[0]), compositing=int(scnt[1]), loss=int(scnt[2])))

    def debug_tiles(self, w, h, capacity, stream=None):
        tx, ty = (w + 15) // 16, (h + 15) // 16
        ranges = torch.zeros((tx * ty, 2), dtype=torch.int32, device="cuda")
        ids = torch.zeros(max(capacity, 1), dtype=torch.int32, device="cuda")
        m = C.c_int64(0)
        self._ok(_lib.gs2_debug_tiles(self.h, _ptr(ranges), _ptr(ids), int(capacity), C.byref(m), _stream(stream)),
                 "gs2_debug_tiles")
        return ranges, ids[: min(m.value, capacity)], m.value

    def debug_lookback_timeout(self, chunk, limit, stream=None):
        """Runs the scan's bounded look-back wait on states nothing publishes (test of the timeout path)."""
        self._ok(_lib.gs2_debug_lookback_timeout(self.h, int(chunk), int(limit), _stream(stream)),
                 "gs2_debug_lookback_timeout")

    def fp64_resolves(self, reset=True):
        """Blocks (colour: channels) re-solved in FP64 per group since the last reset."""
        out = (C.c_uint64 * 5)()
        self._ok(_lib.gs2_fp64_resolves(self.h, out, 1 if reset else 0), "gs2_fp64_resolves")
        return [int(x) for x in out]

    @staticmethod
    def debug_proj(proj, n, stream=None):
        out = torch.empty((DEBUG_PROJ_ROWS, n), dtype=torch.float32, device="cuda")
        keys = torch.empty(n, dtype=torch.int32, device="cuda")
        assert _lib.gs2_debug_proj(_ptr(proj), int(n), _ptr(out), _stream(stream)) == 0
        assert _lib.gs2_debug_keys(_ptr(proj), int(n), _ptr(keys), _stream(stream)) == 0
        return out, keys


def render_noalloc(scene: DeviceScene, cam, proj, image, raster_state, status=None, config: dict | None = None,
                   stream=None):
    """One view rendered without any device allocation by the library (see
    gs2_render_noalloc in include/gs2.h); all buffers are the caller's."""
    cfg = _config_struct(config)
    s = scene.struct()
    st = _lib.gs2_render_noalloc(C.byref(cfg), C.byref(s), C.byref(camera_struct(cam)), _ptr(proj), _ptr(image),
                                 _ptr(raster_state), _ptr(status), _stream(stream))
    if st != 0:
        raise GS2Error(f"gs2_render_noalloc: {STATUS.get(st, st)}")


class Batch:
    """Many independent scenes swept together (include/gs2.h gs2_batch_*).

    sizes: list of dicts with max_gaussians, max_width, max_height,
    max_sh_degree, max_pairs (0 = default) per scene."""

    def __init__(self, sizes, config: dict | None = None):
        self.config = default_config(**(config or {}))
        cfg = _config_struct(self.config)
        desc = (BatchScene_ * len(sizes))(*[BatchScene_(int(d["max_gaussians"]), int(d["max_width"]),
                                                        int(d["max_height"]), int(d.get("max_sh_degree", 3)),
                                                        int(d.get("max_pairs", 0))) for d in sizes])
        h = _vp()
        st = _lib.gs2_batch_create(C.byref(h), C.byref(cfg), len(sizes), desc)
        if st != 0:
            raise GS2Error(f"gs2_batch_create: {STATUS.get(st, st)}")
        self.h = h
        self.n = len(sizes)

    def close(self):
        if getattr(self, "h", None):
            _lib.gs2_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ctx_handle(self, i: int):
        return _lib.gs2_batch_ctx(self.h, int(i))

    def stats(self):
        a, b, r = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        _lib.gs2_batch_stats(self.h, C.byref(a), C.byref(b), C.byref(r))
        return dict(instantiations=a.value, updates=b.value, replays=r.value)

    def set_config(self, i: int, **kw):
        """gs2_set_config on scene i's context (fields not given keep the batch's configuration)."""
        cfg = _config_struct({**self.config, **kw})
        st = _lib.gs2_set_config(self.ctx_handle(i), C.byref(cfg))
        if st != 0:
            raise GS2Error(f"gs2_set_config: {STATUS.get(st, st)}")

    def tuning(self, i: int) -> dict:
        """gs2_get_tuning of scene i's context."""
        t = Tuning_()
        st = _lib.gs2_get_tuning(self.ctx_handle(i), C.byref(t))
        if st != 0:
            raise GS2Error(f"gs2_get_tuning: {STATUS.get(st, st)}")
        return _tuning_dict(t)

    def set_tuning(self, i: int, sort_blocks: int, sort_rows: int, view_lanes: int = 1, accum_px: int = 2,
                   accum_split: int = 0):
        t = Tuning_(int(sort_blocks), int(sort_rows), int(view_lanes), int(accum_px), int(accum_split))
        st = _lib.gs2_set_tuning(self.ctx_handle(i), C.byref(t))
        if st != 0:
            raise GS2Error(f"gs2_set_tuning: {STATUS.get(st, st)}")

    def autotune(self, i: int, scene: DeviceScene, cams, targets, knn, t, reps=2, stream=None):
        """gs2_autotune on scene i's context (a scratch copy of the scene is timed)."""
        arr = (Camera_ * len(cams))(*[camera_struct(c) for c in cams])
        tp = (_vp * len(targets))(*[_ptr(x) for x in targets])
        kt = np.ascontiguousarray(knn, np.int32)
        s = scene.struct()
        best = Tuning_()
        ms = C.c_float(0.0)
        st = _lib.gs2_autotune(self.ctx_handle(i), C.byref(s), arr, len(cams), tp, kt.ctypes.data_as(_vp), int(t),
                               int(reps), C.byref(best), C.byref(ms), _stream(stream))
        if st != 0:
            raise GS2Error(f"gs2_autotune: {STATUS.get(st, st)}")
        return dict(_tuning_dict(best), ms=float(ms.value))

    def prepare(self, scenes, cams, targets, knn):
        """Marshals the per-scene host arrays once (cameras, target pointers,
        KNN tables); the returned object is passed to sweep()."""
        cam_arrs = [(Camera_ * len(c))(*[camera_struct(x) for x in c]) for c in cams]
        tgt_arrs = [(_vp * len(tg))(*[_ptr(x) for x in tg]) for tg in targets]
        knn_arrs = [np.ascontiguousarray(k, np.int32) for k in knn]
        prep = dict(
            scenes=(Scene_ * self.n)(*[s.struct() for s in scenes]),
            cams=(C.POINTER(Camera_) * self.n)(*[C.cast(a, C.POINTER(Camera_)) for a in cam_arrs]),
            ncam=(C.c_int32 * self.n)(*[len(c) for c in cams]),
            tgts=(C.POINTER(_vp) * self.n)(*[C.cast(a, C.POINTER(_vp)) for a in tgt_arrs]),
            knn=(C.POINTER(C.c_int32) * self.n)(*[k.ctypes.data_as(C.POINTER(C.c_int32)) for k in knn_arrs]),
            keep=(cam_arrs, tgt_arrs, knn_arrs, scenes, targets))
        return prep

    def set_targets(self, prep, i: int, targets):
        """Point scene i's target list of a prepared batch at other device
        images (None where a sweep reads none), e.g. per-sweep uploads."""
        arr = prep["keep"][1][i]
        assert len(targets) == len(arr)
        for j, x in enumerate(targets):
            arr[j] = _ptr(x)
        prep["keep"][4][i] = list(targets)

    def sweep(self, prep, t, losses=None, n_failed=None, use_graph=False, stream=None):
        """use_graph: False (eager), True or 1 (one graph, re-captured and
        updated per call), 2 (graphs kept per scene and sweep inputs)."""
        tt = (C.c_int32 * self.n)(*[int(x) for x in t])
        st = _lib.gs2_batch_sweep(self.h, prep["scenes"], prep["cams"], prep["ncam"], prep["tgts"], prep["knn"], tt,
                                  _ptr(losses), _ptr(n_failed), int(use_graph), _stream(stream))
        if st != 0:
            raise GS2Error(f"gs2_batch_sweep: {STATUS.get(st, st)}: {_lib.gs2_batch_last_error(self.h).decode()}")

    def check(self, stream=None):
        torch.cuda.synchronize()
        for i in range(self.n):
            st = _lib.gs2_check(self.ctx_handle(i), _stream(stream))
            if st != 0:
                raise GS2Error(f"scene {i}: {STATUS.get(st, st)}")


class HostTargets:
    """Sweep targets kept in pinned host memory and uploaded per sweep.

    Only the images a sweep reads (its primary and KNN views) are copied, on
    a copy stream, into one of two device buffer sets: the upload of the next
    sweep's views (`prefetch`) runs while the current sweep computes.  A
    buffer set is written again only after the sweep that read it has
    finished on its compute stream (`release`).  Plumbing only: the copies
    are plain host-to-device transfers.

        ht = HostTargets(images, knn)
        for i, t in enumerate(primaries):
            tg = ht.targets(t)                 # device tensors for t's views
            ctx.sweep(scene, cams, tg, knn, t)
            ht.release(t)
            if i + 1 < len(primaries):
                ht.prefetch(primaries[i + 1])
    """

    def __init__(self, images, knn):
        self.host = [im if im.is_pinned() else im.contiguous().pin_memory() for im in images]
        self.knn = np.asarray(knn, np.int32).reshape(len(self.host), -1)
        self.copy = torch.cuda.Stream()
        self.sets = [[], []]
        self.ready = [torch.cuda.Event(), torch.cuda.Event()]
        self.free = [torch.cuda.Event(), torch.cuda.Event()]
        self.used = [False, False]
        self.next_set = 0
        self.pending = {}

    def views(self, t: int):
        return [int(t)] + [int(v) for v in self.knn[t] if v >= 0]

    def bytes_for(self, t: int) -> int:
        return sum(self.host[v].numel() * self.host[v].element_size() for v in self.views(t))

    def prefetch(self, t: int):
        """Enqueue the upload of sweep t's views on the copy stream."""
        t = int(t)
        if t in self.pending:
            return
        s = self.next_set
        self.next_set ^= 1
        views = self.views(t)
        bufs = self.sets[s]
        while len(bufs) < len(views):
            bufs.append(None)
        with torch.cuda.stream(self.copy):
            if self.used[s]:
                self.copy.wait_event(self.free[s])
            for j, v in enumerate(views):
                src = self.host[v]
                if bufs[j] is None or bufs[j].shape != src.shape or bufs[j].dtype != src.dtype:
                    bufs[j] = torch.empty(src.shape, dtype=src.dtype, device="cuda")
                bufs[j].copy_(src, non_blocking=True)
            self.ready[s].record(self.copy)
        self.pending[t] = s

    def targets(self, t: int, stream=None):
        """Target list for sweep t: device tensors at its views, None
        elsewhere (a sweep reads no other entry); `stream` (default: the
        current one) waits for the upload."""
        t = int(t)
        self.prefetch(t)
        s = self.pending[t]
        (stream or torch.cuda.current_stream()).wait_event(self.ready[s])
        tg = [None] * len(self.host)
        for j, v in enumerate(self.views(t)):
            tg[v] = self.sets[s][j]
        return tg

    def release(self, t: int, stream=None):
        """Mark sweep t's buffer set free once the work enqueued so far on
        `stream` (its sweep) has run."""
        s = self.pending.pop(int(t))
        self.free[s].record(stream or torch.cuda.current_stream())
        self.used[s] = True


def _mlp_call(st, what):
    if st != 0:
        raise GS2Error(f"{what}: {STATUS.get(st, st)}")


def mlp_forward(w_bf16, records, chunk_n, nrec, idx=None, out=None, stream=None):
    """alpha of records (chunks [REC_ROWS][chunk_n]); out: device float [nrec]."""
    if out is None:
        out = torch.empty(max(int(nrec), 1), dtype=torch.float32, device="cuda")
    _mlp_call(_lib.gs2_mlp_forward(_ptr(w_bf16), _ptr(records), int(chunk_n), _ptr(idx), int(nrec), _ptr(out),
                                   _stream(stream)), "gs2_mlp_forward")
    return out[: int(nrec)]


def mlp_grad(w_bf16, records, chunk_n, nrec, partial, stats, idx=None, chunk_scale=None, stream=None):
    """Per-CTA gradient sums [MLP_GRID][MLP_NPARAM] and (loss, count) [MLP_GRID][2];
    with chunk_scale the line-model loss, else the label loss."""
    _mlp_call(_lib.gs2_mlp_grad(_ptr(w_bf16), _ptr(records), int(chunk_n), _ptr(idx), int(nrec), _ptr(chunk_scale),
                                _ptr(partial), _ptr(stats), _stream(stream)), "gs2_mlp_grad")


def records_chunk_scale(records, chunk_n, n_chunks, out=None, stream=None):
    if out is None:
        out = torch.empty(max(int(n_chunks), 1), dtype=torch.float32, device="cuda")
    _mlp_call(_lib.gs2_records_chunk_scale(_ptr(records), int(chunk_n), int(n_chunks), _ptr(out), _stream(stream)),
              "gs2_records_chunk_scale")
    return out[: int(n_chunks)]


def mlp_adam(master, w_bf16, partial, stats, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _mlp_call(_lib.gs2_mlp_adam(_ptr(master), _ptr(w_bf16), _ptr(partial), _ptr(stats), _ptr(m), _ptr(v),
                                int(step), float(lr), float(beta1), float(beta2), float(eps), _stream(stream)),
              "gs2_mlp_adam")


def launch_count() -> int:
    return int(_lib.gs2_launch_count())


def camera_knn(centres: np.ndarray, sphere: np.ndarray, k: int) -> np.ndarray:
    c = np.ascontiguousarray(centres, np.float32)
    s = np.ascontiguousarray(sphere, np.float32)
    out = np.zeros((c.shape[0], k), np.int32)
    st = _lib.gs2_camera_knn(c.ctypes.data_as(_vp), c.shape[0], s.ctypes.data_as(_vp), int(k),
                             out.ctypes.data_as(_vp))
    if st != 0:
        raise GS2Error(f"gs2_camera_knn: {STATUS.get(st, st)}")
    return out
