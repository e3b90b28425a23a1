"""The C-ABI library loads, exports every symbol include/*.h declares, and
rejects bad arguments before touching the GPU (host-side checks only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SO = os.path.join(ROOT, "paper_1412_1945_gb300", "libocq.so")


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ocq_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(SO):
        from paper_1412_1945_gb300 import _build

        _build.build()
    import paper_1412_1945_gb300 as ocq

    return ocq.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "ocq_build_model" in names and "ocq_classify" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib):
    from paper_1412_1945_gb300 import ocq

    for n in declared_functions():
        assert n in ocq.SIGNATURES, n
        assert hasattr(ocq, n), n


def test_host_side_helpers(lib):
    from paper_1412_1945_gb300 import ocq

    assert ocq.ocq_status_str(0) == "OCQ_OK"
    assert ocq.ocq_status_str(4) == "OCQ_ETIMEOUT"
    assert ocq.ocq_region_count(1080, 1920, ocq.OCQ_REGION_PIXEL) == 1920 * 1080
    assert ocq.ocq_region_count(240, 320, ocq.OCQ_REGION_BLOCK, 16) == 300
    assert ocq.ocq_region_count(241, 321, ocq.OCQ_REGION_BLOCK, 16) == 16 * 21
    assert ocq.ocq_region_count(10, 10, ocq.OCQ_REGION_BLOCK, 0) == -1
    assert ocq.ocq_region_count(0, 10, ocq.OCQ_REGION_FRAME) == -1
    # model bytes: regions x max(1, 8^d / 32) u32 words
    assert ocq.ocq_model_footprint(1080, 1920, ocq.OCQ_REGION_PIXEL, 0, 3) == 1920 * 1080 * 64
    assert ocq.ocq_model_footprint(240, 320, ocq.OCQ_REGION_BLOCK, 16, 5) == 300 * 4096
    # per-pixel depth 4-5: plus the kept-leaf index, 8 u16 codes per location
    assert ocq.ocq_model_footprint(1080, 1920, ocq.OCQ_REGION_PIXEL, 0, 4) == 1920 * 1080 * (512 + 16)
    assert ocq.ocq_model_footprint(1080, 1920, ocq.OCQ_REGION_PIXEL, 0, 6) == 1920 * 1080 * 32768
    assert ocq.ocq_model_footprint(120, 160, ocq.OCQ_REGION_FRAME, 0, 1) == 4
    assert ocq.ocq_model_footprint(120, 160, ocq.OCQ_REGION_FRAME, 0, 9) == 0


def test_camera_footprint_follows_the_model_form(lib):
    """A camera reserves the model in the form ocq_build_model gives its
    description and its window: per-pixel d = 5 with floor(N/T) <= 8 is a
    list model (16 B per location), with floor(N/T) > 8 rows (4 KB per
    location), and with list models switched off rows plus the lists; pixel
    cameras of depth <= 5 keep 2-byte leaf codes per pixel and frame and merge
    in place (one model), depth 6 keeps the frames and a second model; a
    whole-frame camera keeps N leaf bitsets and per-leaf u16 counts."""
    from paper_1412_1945_gb300 import ocq

    H, W, N, K = 1080, 1920, 30, 30
    hw, codes, frames = H * W, N * H * W * 2, N * H * W * 3
    pix = ocq.OCQ_REGION_PIXEL
    assert ocq.ocq_server_camera_footprint(H, W, pix, 0, 5, 10, N, K) == hw * 16 + codes
    assert ocq.ocq_server_camera_footprint(H, W, pix, 0, 5, 3, N, K) == hw * 4096 + codes
    assert ocq.ocq_server_camera_footprint(H, W, pix, 0, 3, 10, N, K) == hw * 64 + codes
    assert ocq.ocq_server_window_bytes(H, W, pix, 0, 3, 10, N, K) == codes
    # depth 6: two models of 8^6 bits per location, the frames, and the build's
    # chunk scratch (8^(d-3)/8 bytes per location)
    assert ocq.ocq_server_camera_footprint(64, 64, pix, 0, 6, 10, N, K) == 2 * (64 * 64 * 8 ** 6 // 8) + \
        N * 64 * 64 * 3 + 64 * 64 * 8 ** 3 // 8
    fr = ocq.OCQ_REGION_FRAME
    wb = 8 ** 4 // 8
    assert ocq.ocq_server_camera_footprint(H, W, fr, 0, 4, 10, N, K) == wb + N * wb + N * wb + 2 * 8 ** 4 + N * wb
    assert ocq.ocq_server_window_bytes(H, W, fr, 0, 4, 10, N, K) == N * wb
    assert ocq.ocq_server_window_bytes(8, 8, fr, 0, 6, 10, N, K) == N * 8 * 8 * 3  # bitset larger than a frame
    mf = ocq.OCQ_TUNE_PIXEL_MODEL_FORM
    saved = ocq.ocq_tune_selected(mf)
    try:
        ocq.ocq_tune_select(mf, 0)
        assert ocq.ocq_server_camera_footprint(H, W, pix, 0, 5, 10, N, K) == hw * (4096 + 16) + codes
    finally:
        ocq.ocq_tune_select(mf, saved)


@pytest.mark.parametrize("N,H,W,kind,block,depth,T", [
    (0, 8, 8, 0, 0, 3, 1),      # N < 1
    (4, 8, 8, 0, 0, 3, 5),      # T > N
    (4, 8, 8, 0, 0, 3, 0),      # T < 1
    (4, 8, 8, 0, 0, 0, 1),      # depth < 1
    (4, 8, 8, 0, 0, 9, 1),      # depth > 8
    (4, 0, 8, 0, 0, 3, 1),      # H < 1
    (4, 8, 8, 1, 0, 3, 1),      # block < 1
    (4, 8, 8, 7, 0, 3, 1),      # unknown region kind
    (70000, 8, 8, 0, 0, 3, 1),  # N > 65535
])
def test_build_rejects_bad_arguments(lib, N, H, W, kind, block, depth, T):
    from paper_1412_1945_gb300 import ocq

    with pytest.raises(ocq.OcqError) as e:
        ocq.ocq_build_model(0x1000, N, H, W, kind, block, depth, T, stream=0)
    assert e.value.status == ocq.OCQ_EINVAL
    assert ocq.ocq_last_error()


def test_null_pointers_rejected(lib):
    from paper_1412_1945_gb300 import ocq

    with pytest.raises(ocq.OcqError) as e:
        ocq.ocq_build_model(None, 4, 8, 8, 0, 0, 3, 2, stream=0)
    assert e.value.status == ocq.OCQ_EINVAL
    with pytest.raises(ocq.OcqError) as e:
        ocq.ocq_classify(None, 0x1000, 1, 0x2000, stream=0)
    assert e.value.status == ocq.OCQ_EINVAL
    with pytest.raises(ocq.OcqError) as e:
        ocq.ocq_path_code(None, 10, 3, 0x1000, stream=0)
    assert e.value.status == ocq.OCQ_EINVAL
    with pytest.raises(ocq.OcqError) as e:
        ocq.ocq_path_code(0x1000, 10, 0, 0x1000, stream=0)
    assert e.value.status == ocq.OCQ_EINVAL
    with pytest.raises(ocq.OcqError) as e:
        ocq.ocq_model_export(None, 0x1000, 1, stream=0)
    assert e.value.status == ocq.OCQ_EINVAL
    with pytest.raises(ocq.OcqError) as e:
        ocq.ocq_occupancy(0x1000, 1, 8, 8, 1, 0, 3, 0x1000, stream=0)
    assert e.value.status == ocq.OCQ_EINVAL
    # zero-size work is a no-op that touches nothing
    ocq.ocq_path_code(None, 0, 3, None, stream=0)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1412_1945_gb300 import ocq

    saved = ocq._lib
    try:
        ocq._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            ocq.load(str(tmp_path / "absent.so"))
    finally:
        ocq._lib = saved
