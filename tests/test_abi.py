"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
function include/krig.h declares, and the planner validates its arguments."""
import ctypes
import os
import re

import pytest

from paper_2303_09523_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(krig_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return binding.lib(build_if_missing=True)


def test_header_declares_entry_points():
    names = _declared_functions()
    for n in ("krig_plan_create", "krig_plan_set_workspace", "krig_interpolate", "krig_plan_device_status",
              "krig_last_error", "krig_plan_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared_functions():
        assert hasattr(lib, n), "libkrig.so does not export %s" % n


def test_version(lib):
    assert lib.krig_version() >= 100


def _desc(**kw):
    d = dict(H=64, W=64, n_known=9, zfactor=4, n_sub_blocks=2, half_w=1, in_dtype=binding.F64, in_scale=1.0)
    d.update(kw)
    return d


def _create(descs, form=binding.FORM_DS, flags=0):
    L = binding.lib()
    arr = (binding.VolumeDesc * max(1, len(descs)))()
    for i, d in enumerate(descs):
        arr[i] = binding.VolumeDesc(d["H"], d["W"], d["n_known"], d["zfactor"], d["n_sub_blocks"], d["half_w"],
                                    d["in_dtype"], d["in_scale"])
    h = ctypes.c_void_p()
    nb = ctypes.c_size_t()
    st = L.krig_plan_create(ctypes.byref(h), arr, len(descs), form, flags, ctypes.byref(nb))
    return st, h, nb.value


@pytest.mark.parametrize("form", [binding.FORM_DS, binding.FORM_P64, binding.FORM_PMX])
def test_plan_create_and_workspace_size(lib, form):
    st, h, nb = _create([_desc(), _desc(H=37, W=45, n_known=5, zfactor=3, half_w=2, in_dtype=binding.F32)], form)
    assert st == binding.KRIG_OK
    assert nb >= 256 and nb % 256 == 0
    lib.krig_plan_destroy(h)


@pytest.mark.parametrize("bad,status", [
    (dict(H=0), binding.KRIG_EINVAL),
    (dict(W=70000), binding.KRIG_EINVAL),
    (dict(n_known=1), binding.KRIG_EINVAL),
    (dict(zfactor=0), binding.KRIG_EINVAL),
    (dict(zfactor=9), binding.KRIG_EINVAL),
    (dict(n_sub_blocks=0), binding.KRIG_EINVAL),
    (dict(n_sub_blocks=9), binding.KRIG_EINVAL),   # more blocks than gaps
    (dict(half_w=3), binding.KRIG_EUNSUPPORTED),
    (dict(in_dtype=7), binding.KRIG_EINVAL),
    (dict(in_dtype=binding.U16, in_scale=0.0), binding.KRIG_EINVAL),
])
def test_plan_create_rejects(lib, bad, status):
    st, h, _ = _create([_desc(**bad)])
    assert st == status
    assert h.value is None
    assert len(lib.krig_last_error()) > 0


def test_plan_create_limits(lib):
    assert _create([])[0] == binding.KRIG_EINVAL
    assert _create([_desc()] * 65)[0] == binding.KRIG_EINVAL
    st, h, _ = _create([_desc()] * 64)
    assert st == binding.KRIG_OK
    lib.krig_plan_destroy(h)
    assert _create([_desc()], form=9)[0] == binding.KRIG_EINVAL
    assert _create([_desc()], flags=0x80)[0] == binding.KRIG_EINVAL


def test_calls_without_workspace_are_rejected(lib):
    st, h, _ = _create([_desc()])
    assert st == binding.KRIG_OK
    p = (ctypes.c_void_p * 1)(16)
    assert lib.krig_interpolate(h, p, p, None, ctypes.c_void_p(16), None) == binding.KRIG_EWORKSPACE
    assert lib.krig_plan_set_workspace(h, None, 1 << 20) == binding.KRIG_EWORKSPACE
    assert lib.krig_plan_set_workspace(h, ctypes.c_void_p(256 + 8), 1 << 20) == binding.KRIG_EWORKSPACE
    assert lib.krig_plan_set_workspace(h, ctypes.c_void_p(256), 8) == binding.KRIG_EWORKSPACE
    lib.krig_plan_destroy(h)
    lib.krig_plan_destroy(None)


def test_null_plan(lib):
    assert lib.krig_interpolate(None, None, None, None, None, None) == binding.KRIG_EINVAL
    assert lib.krig_plan_device_status(None, None) == binding.KRIG_EINVAL


@pytest.mark.parametrize("bad,lag", [
    (dict(), 17),                                   # lag beyond the halo the kernel stages
    (dict(), -1),
    (dict(H=0), 2),
    (dict(n_known=0), 2),
    (dict(in_dtype=7), 2),
    (dict(in_dtype=binding.U16, in_scale=-1.0), 2),
])
def test_empirical_variogram_rejects_before_any_launch(lib, bad, lag):
    d = _desc(**bad)
    vd = binding.VolumeDesc(d["H"], d["W"], d["n_known"], d["zfactor"], d["n_sub_blocks"], d["half_w"],
                            d["in_dtype"], d["in_scale"])
    counts = (ctypes.c_int64 * 2)()
    st = lib.krig_empirical_variogram(ctypes.byref(vd), ctypes.c_void_p(256), lag, ctypes.c_void_p(256), counts,
                                      None)
    assert st == binding.KRIG_EINVAL
    assert len(lib.krig_last_error()) > 0
    assert lib.krig_empirical_variogram(None, ctypes.c_void_p(256), 2, ctypes.c_void_p(256), None,
                                        None) == binding.KRIG_EINVAL
    assert lib.krig_empirical_variogram(ctypes.byref(vd), None, 2, ctypes.c_void_p(256), None,
                                        None) == binding.KRIG_EINVAL


@pytest.mark.parametrize("bad,status", [
    (dict(H=0), binding.KRIG_EINVAL),
    (dict(n_known=1), binding.KRIG_EINVAL),
    (dict(zfactor=9), binding.KRIG_EINVAL),
    (dict(n_sub_blocks=9), binding.KRIG_EINVAL),
    (dict(half_w=3), binding.KRIG_EUNSUPPORTED),
    (dict(in_dtype=7), binding.KRIG_EINVAL),
    (dict(in_dtype=binding.U16, in_scale=0.0), binding.KRIG_EINVAL),
])
def test_noalloc_rejects_what_plan_create_rejects(lib, bad, status):
    """The allocation-free entry point checks a descriptor with the planner's own check,
    before any CUDA call, and returns the same status."""
    d = _desc(**bad)
    vd = binding.VolumeDesc(d["H"], d["W"], d["n_known"], d["zfactor"], d["n_sub_blocks"], d["half_w"],
                            d["in_dtype"], d["in_scale"])
    fn = lib.krig_interpolate_noalloc
    fn.argtypes = [ctypes.POINTER(binding.VolumeDesc), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    st = fn(ctypes.byref(vd), 256, 256, None, 256, 1, None)
    assert st == status == _create([d])[0]
    assert len(lib.krig_last_error()) > 0


def test_similarity_rejects_before_any_launch(lib):
    vp = ctypes.c_void_p
    out = vp(256)
    assert lib.krig_similarity(None, vp(256), 1, 4, 4, vp(256), 1 << 20, out, None) == binding.KRIG_EINVAL
    assert lib.krig_similarity(vp(256), vp(256), 0, 4, 4, vp(256), 1 << 20, out, None) == binding.KRIG_EINVAL
    assert lib.krig_similarity(vp(256), vp(256), 1, 0, 4, vp(256), 1 << 20, out, None) == binding.KRIG_EINVAL
    need = lib.krig_similarity_workspace_bytes(3, 64, 64)
    assert need >= 3 * 256 * 256 * 4
    assert lib.krig_similarity(vp(256), vp(256), 3, 64, 64, vp(256), need - 1, out, None) == binding.KRIG_EWORKSPACE
    assert lib.krig_similarity(vp(256), vp(256), 3, 64, 64, vp(264), need, out, None) == binding.KRIG_EWORKSPACE
    assert lib.krig_similarity_workspace_bytes(0, 4, 4) == 0
