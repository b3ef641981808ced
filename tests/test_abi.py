"""The C-ABI library loads without a GPU and exports every entry point that
include/gs2.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_2501_13975_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gs2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs2_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2501_13975_b300 import gs2
    assert set(declared_symbols()) == set(gs2.EXPORTED)


def test_config_defaults_and_sizes():
    from paper_2501_13975_b300 import gs2
    d = gs2.default_config()
    assert d["ssim_radius"] == 5 and d["knn_k"] == 3 and abs(d["alpha_min"] - 1 / 255) < 1e-9
    lib = gs2._lib
    assert lib.gs2_blocks_bytes(gs2.POS, 10, 3, 4) == 9 * 10 * 4
    assert lib.gs2_blocks_bytes(gs2.COLOR, 10, 3, 4) == (6 + 16) * 10 * 4 * 4
    assert lib.gs2_step_bytes(gs2.COLOR, 10, 3) == 3 * 16 * 10 * 4
    assert lib.gs2_proj_bytes(1000) >= 68 * 1000


def test_camera_knn_host():
    """Host KNN of the library on the ring with known neighbours (same case as
    the oracle pin)."""
    import numpy as np
    from paper_2501_13975_b300 import gs2
    ang = np.radians([0, 10, 30, 60, 100, 150, 210, 280])
    cen = np.stack([5 * np.cos(ang), np.zeros_like(ang), 5 * np.sin(ang)], 1)
    out = gs2.camera_knn(cen, np.array([0, 0, 0, 5.0]), 3)
    assert list(out[0]) == [1, 2, 3] and list(out[7]) == [6, 0, 1]


def test_create_without_device_fails_cleanly():
    """Without a CUDA device gs2_create reports an error instead of crashing."""
    import torch
    if torch.cuda.is_available():
        return
    from paper_2501_13975_b300 import gs2
    try:
        gs2.Context(100, 64, 64, 0)
    except gs2.GS2Error:
        return
    raise AssertionError("expected GS2Error")


def test_create_rejects_shapes_beyond_the_tile_coordinates():
    """A side longer than 65,535 tiles of 16 pixels cannot be binned (tile
    coordinates are 16-bit): gs2_create refuses it before any device call."""
    lib = ctypes.CDLL(B.build())
    lib.gs2_create.restype = ctypes.c_int
    lib.gs2_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                               ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
    h = ctypes.c_void_p()
    shape_err = 2
    for w, hh in ((0xFFFF * 16 + 1, 1), (1, 0xFFFF * 16 + 1), (1 << 15, (1 << 13) + 1)):
        assert lib.gs2_create(ctypes.byref(h), None, 100, w, hh, 0, 0) == shape_err, (w, hh)
        assert not h.value


def test_render_noalloc_refuses_a_bad_config_before_any_device_call():
    """gs2_render_noalloc validates a caller's configuration exactly as
    gs2_create does (alpha_min must lie in (0, 1), near_z > 0, ...) and returns
    GS2_ERR_ARG before it touches a device; the pointers below are never
    dereferenced, so this runs without a GPU."""
    import ctypes as C

    from paper_2501_13975_b300 import gs2
    lib = gs2._lib
    fake = 0x1000
    scene = gs2.Scene_(10, 0, fake, fake, fake, fake, fake)
    cam = gs2.Camera_()
    cam.width, cam.height, cam.fx, cam.fy = 64, 64, 50.0, 50.0
    for field, value in (("alpha_min", 0.0), ("alpha_min", float("nan")), ("near_z", 0.0), ("near_z", -1.0)):
        cfg = gs2._config_struct({field: value})
        st = lib.gs2_render_noalloc(C.byref(cfg), C.byref(scene), C.byref(cam), fake, fake, fake, None, None)
        assert st == 1, (field, value, st)   # GS2_ERR_ARG


def test_model_setters_refuse_a_null_context():
    """gs2_set_step_model and gs2_set_damping_model answer GS2_ERR_ARG for a
    NULL context (host check, no device call)."""
    from paper_2501_13975_b300 import gs2
    for name in ("gs2_set_step_model", "gs2_set_damping_model"):
        f = getattr(gs2._lib, name)
        assert f(None, None) == 1, name


def _header_structs():
    """Field (name, byte size) lists of the anonymous typedef structs in gs2.h, by typedef name."""
    src = open(os.path.join(ROOT, "include", "gs2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    size = {"int32_t": 4, "uint32_t": 4, "float": 4, "int64_t": 8, "double": 8}
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(gs2_[a-z_]+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            m = re.match(r"(\w+)\s*(\*?)\s*(.*)", decl)
            ctype, ptr, names = m.group(1), m.group(2), m.group(3)
            for nm in names.split(","):
                nm = nm.strip()
                star = ptr or nm.startswith("*")
                nm = nm.lstrip("*").strip()
                arr = re.match(r"(\w+)\[(\d+)\]", nm)
                count = int(arr.group(2)) if arr else 1
                nm = arr.group(1) if arr else nm
                fields.append((nm, (8 if star else size[ctype]) * count))
        out[name] = fields
    return out


def test_binding_structs_match_header():
    """The binding's ctypes structures have the header's fields, in order and
    with the same sizes (a field added on one side only would shift the rest)."""
    import ctypes as C

    from paper_2501_13975_b300 import gs2
    hs = _header_structs()
    pairs = {"gs2_tuning": gs2.Tuning_, "gs2_config": gs2.Config_, "gs2_camera": gs2.Camera_,
             "gs2_scene": gs2.Scene_, "gs2_batch_scene": gs2.BatchScene_}
    for cname, pyt in pairs.items():
        assert cname in hs, cname
        py = [(n, C.sizeof(t)) for n, t in pyt._fields_]
        assert py == hs[cname], (cname, py, hs[cname])
