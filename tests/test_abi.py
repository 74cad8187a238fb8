"""The C-ABI library builds, loads without a GPU, exports every function that
include/gsc.h declares, and rejects bad arguments on the host before any CUDA
call.  No compute call is made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsc.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsc_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2507_19718_gb300 import build, gsc
    build.build()
    return gsc.lib()


def test_every_declared_symbol_is_exported(L):
    from paper_2507_19718_gb300 import gsc
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(gsc.SIGNATURES) == names


def test_version_and_lr_schedule(L, orc):
    assert L.gsc_abi_version() == 1
    for t in [0, 1, 2, 3, 10, 100, 12345]:
        assert L.gsc_lr_scale(t) == pytest.approx(orc.lr_scale(max(t, 1)), rel=1e-7)


def test_workspace_size_grows_with_limits(L):
    from paper_2507_19718_gb300 import gsc
    def size(*a):
        n = C.c_size_t()
        assert L.gsc_workspace_size(*a, 1, None, C.byref(n)) == 0
        return n.value
    a = size(1024, 100000, 128, 128)
    b = size(2048, 100000, 128, 128)
    c = size(1024, 200000, 128, 128)
    d = size(1024, 100000, 1920, 1080)
    assert 0 < a < b and a < c and a < d and a % 256 == 0
    # 4 arrays of 4-byte (key, value) per pair
    assert c - a >= 100000 * 16 - 4 * 256
    n = C.c_size_t()
    assert L.gsc_workspace_size(-1, 10, 8, 8, 1, None, C.byref(n)) == gsc.GSC_ERR_INVALID_ARG
    assert L.gsc_workspace_size(10, 10, 8, 8, 33, None, C.byref(n)) == gsc.GSC_ERR_INVALID_ARG
    n4 = C.c_size_t()
    assert L.gsc_workspace_size(1024, 100000, 128, 128, 4, None, C.byref(n4)) == 0
    assert n4.value > a


def test_host_side_validation(L):
    from paper_2507_19718_gb300 import gsc
    # scene: grid too small
    d = gsc.SceneDesc()
    d.nx, d.ny, d.nz = 1, 8, 8
    d.density = 0x1000
    d.density_max, d.sigma_max, d.albedo, d.tf_count = 20.0, 20.0, 0.8, 2
    d.tf_pos[:2] = [0.0, 1.0]
    h = C.c_void_p()
    assert L.gsc_scene_create(C.byref(d), C.byref(h)) == gsc.GSC_ERR_INVALID_ARG
    buf = C.create_string_buffer(256)
    L.gsc_last_error(buf, 256)
    assert b"grid" in buf.value
    # a valid descriptor creates a host-only handle (nothing is enqueued)
    d.nx = 8
    assert L.gsc_scene_create(C.byref(d), C.byref(h)) == 0
    pos = (C.c_float * 2)(0.5, 0.2)
    rgba = (C.c_float * 8)(*([0.5] * 8))
    assert L.gsc_scene_set_tf(h, 2, pos, rgba) == gsc.GSC_ERR_INVALID_ARG  # not ascending
    assert L.gsc_scene_destroy(h) == 0
    # workspace: unaligned buffer / too small
    w = C.c_void_p()
    assert L.gsc_workspace_create(C.c_void_p(0x1001), 1 << 30, 16, 16, 8, 8, 1, None, C.byref(w)) == \
        gsc.GSC_ERR_INVALID_ARG
    assert L.gsc_workspace_create(C.c_void_p(0x1000), 16, 16, 16, 8, 8, 1, None, C.byref(w)) == gsc.GSC_ERR_OOM
    # batch: too many views, bad mode
    views = (gsc.View * 2)()
    cfg0 = gsc.raster_cfg()
    assert L.gsc_render_batch(views, 33, 1, C.byref(cfg0), None, None) == gsc.GSC_ERR_INVALID_ARG
    assert L.gsc_render_batch(views, 2, 4, C.byref(cfg0), None, None) == gsc.GSC_ERR_INVALID_ARG
    tviews = (gsc.TrainView * 2)()
    assert L.gsc_train_batch(tviews, 0, 0, C.byref(cfg0), None, None) == gsc.GSC_ERR_INVALID_ARG
    assert L.gsc_train_batch(tviews, 2, gsc.LOSS_L1_SSIM, C.byref(cfg0), None, None) == gsc.GSC_ERR_INVALID_ARG
    # fused training step: adam, m and v are required
    mv = (C.c_void_p * 2)(256, 256)
    a1 = gsc.adam_params([0.01] * 16)
    assert L.gsc_train_step(tviews, mv, mv, 2, gsc.LOSS_HDR, None, C.byref(cfg0), None, None) == \
        gsc.GSC_ERR_INVALID_ARG
    assert L.gsc_train_step(tviews, None, mv, 2, gsc.LOSS_HDR, C.byref(a1), C.byref(cfg0), None, None) == \
        gsc.GSC_ERR_INVALID_ARG
    assert L.gsc_train_step(tviews, mv, mv, 0, gsc.LOSS_HDR, C.byref(a1), C.byref(cfg0), None, None) == \
        gsc.GSC_ERR_INVALID_ARG
    # render: bad tile shape, then NULL workspace
    cam = gsc.Camera()
    cam.fx = cam.fy = 100.0
    cam.width = cam.height = 32
    cfg = gsc.raster_cfg(tile=(12, 12))
    assert L.gsc_cache_render(None, 0, C.byref(cam), C.byref(cfg), None, None, None) == gsc.GSC_ERR_INVALID_ARG
    cfg = gsc.raster_cfg(tile=(16, 16), list_capacity=100)
    assert L.gsc_cache_render(None, 0, C.byref(cam), C.byref(cfg), None, None, None) == gsc.GSC_ERR_INVALID_ARG
    cfg = gsc.raster_cfg()
    assert L.gsc_cache_render(None, 0, C.byref(cam), C.byref(cfg), None, None, None) == gsc.GSC_ERR_INVALID_ARG
    # pixels per thread: only the compiled (tile, ppt) pairs pass the configuration check
    msg = C.create_string_buffer(256)
    for tile, ppt, ok in [((16, 16), 8, True), ((8, 32), 4, True), ((32, 8), 2, True), ((8, 8), 4, False),
                          ((16, 16), 3, False), ((32, 4), 2, False), ((16, 16), 16, False)]:
        cfg = gsc.raster_cfg(tile=tile, pixels_per_thread=ppt)
        assert L.gsc_cache_render(None, 0, C.byref(cam), C.byref(cfg), None, None, None) == gsc.GSC_ERR_INVALID_ARG
        L.gsc_last_error(msg, 256)
        assert (b"pixels per thread" not in msg.value) == ok, (tile, ppt, msg.value)
    # optimiser: bad hyper-parameters
    a = gsc.adam_params([0.01] * 16, step=0)
    assert L.gsc_cache_step(C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), C.c_void_p(256), 4, C.byref(a),
                            None) == gsc.GSC_ERR_INVALID_ARG
    # loss: kind not available / crop outside
    assert L.gsc_loss(7, C.c_void_p(256), C.c_void_p(256), 3, 8, 8, None, None, C.c_void_p(256), C.c_void_p(256),
                      None) == gsc.GSC_ERR_INVALID_ARG
    # a crop whose end overflows 32-bit int is rejected before any launch, with and without a workspace
    big = (C.c_int32 * 4)(2 ** 31 - 1, 0, 1, 8)
    tall = (C.c_int32 * 4)(0, 2 ** 31 - 4, 8, 8)
    for crop in (big, tall):
        assert L.gsc_loss(0, C.c_void_p(256), C.c_void_p(256), 3, 8, 8, crop, C.c_void_p(256), C.c_void_p(256),
                          C.c_void_p(256), None) == gsc.GSC_ERR_INVALID_ARG
        assert L.gsc_loss_noalloc(0, C.c_void_p(256), C.c_void_p(256), 3, 8, 8, crop, C.c_void_p(256),
                                  C.c_void_p(256), None) == gsc.GSC_ERR_INVALID_ARG
        L.gsc_last_error(msg, 256)
        assert b"crop" in msg.value
