"""Thin ctypes binding of ``libocq.so`` (``include/ocq.h``).

Functions keep the C names and argument order.  Pointer arguments accept a
CUDA tensor (its ``data_ptr()``), a plain integer address, or None.  A
``stream`` argument accepts a ``torch.cuda.Stream``, a raw ``cudaStream_t``
integer, or None for the current torch stream.  Non-OK statuses raise
``OcqError``.  Every computation runs in the CUDA library; there is no other
code path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "libocq.so")

OCQ_OK, OCQ_EINVAL, OCQ_ENOMEM, OCQ_ECUDA, OCQ_ETIMEOUT, OCQ_EBUSY, OCQ_ENOTSUP = range(7)
OCQ_REGION_FRAME, OCQ_REGION_BLOCK, OCQ_REGION_PIXEL = 0, 1, 2

_lock = threading.Lock()
_lib = None


class OcqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


STATUS_NAMES = {0: "OCQ_OK", 1: "OCQ_EINVAL", 2: "OCQ_ENOMEM", 3: "OCQ_ECUDA", 4: "OCQ_ETIMEOUT",
                5: "OCQ_EBUSY", 6: "OCQ_ENOTSUP"}


class ocq_region(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("block", ctypes.c_int32)]


class ocq_model_info(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("region_kind", ctypes.c_int32),
                ("block", ctypes.c_int32), ("depth", ctypes.c_int32), ("T", ctypes.c_int32),
                ("N", ctypes.c_int32), ("reserved", ctypes.c_int32), ("regions", ctypes.c_int64),
                ("words_per_region", ctypes.c_int64)]


class ocq_stream_desc(ctypes.Structure):
    _fields_ = [("train", ctypes.c_void_p), ("N", ctypes.c_int), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("region", ocq_region), ("depth", ctypes.c_int), ("T", ctypes.c_int), ("test", ctypes.c_void_p),
                ("F", ctypes.c_int), ("mask", ctypes.c_void_p)]


class ocq_camera_desc(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("region", ocq_region), ("depth", ctypes.c_int),
                ("T", ctypes.c_int), ("N", ctypes.c_int), ("K", ctypes.c_int)]


class ocq_completion(ctypes.Structure):
    _fields_ = [("camera", ctypes.c_int32), ("reserved", ctypes.c_int32), ("frame", ctypes.c_int64),
                ("tag", ctypes.c_uint64), ("arrival_s", ctypes.c_double), ("done_s", ctypes.c_double)]


# name -> (restype, argtypes)
_vp, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "ocq_status_str": (ctypes.c_char_p, [_i32]),
    "ocq_last_error": (ctypes.c_char_p, []),
    "ocq_version": (ctypes.c_char_p, []),
    "ocq_region_count": (_i64, [_i32, _i32, ocq_region]),
    "ocq_model_footprint": (_sz, [_i32, _i32, ocq_region, _i32]),
    "ocq_path_code": (_i32, [_vp, _i64, _i32, _vp, _vp]),
    "ocq_occupancy": (_i32, [_vp, _i32, _i32, _i32, ocq_region, _i32, _vp, _vp]),
    "ocq_build_model": (_i32, [_vp, _i32, _i32, _i32, ocq_region, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "ocq_classify": (_i32, [_vp, _vp, _i32, _vp, _vp]),
    "ocq_model_get_info": (_i32, [_vp, ctypes.POINTER(ocq_model_info)]),
    "ocq_model_export": (_i32, [_vp, _vp, _sz, _vp]),
    "ocq_model_import": (_i32, [_vp, ctypes.POINTER(ocq_model_info), _vp, ctypes.POINTER(_vp)]),
    "ocq_model_free": (None, [_vp]),
    "ocq_device_status": (_i32, [_vp]),
    "ocq_detect_host": (_i32, [_vp, _i32, _vp, _i32, _i32, _i32, ocq_region, _i32, _i32, _vp, _vp,
                               ctypes.POINTER(_vp)]),
    "ocq_kernel_launches": (ctypes.c_uint64, []),
    "ocq_merge_occupancy": (_i32, [_vp, _i32, _i32, _i32, _i32, ocq_region, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "ocq_build_frame_noalloc": (_i32, [_vp, _i32, _i32, _i32, _i32, _i32, _vp, _vp]),
    "ocq_batch_create": (_i32, [ctypes.POINTER(ocq_stream_desc), _i32, _vp, ctypes.POINTER(_vp)]),
    "ocq_batch_run": (_i32, [_vp, _vp]),
    "ocq_batch_status": (_i32, [_vp, _vp]),
    "ocq_batch_model": (_i32, [_vp, _i32, ctypes.POINTER(_vp)]),
    "ocq_batch_set_work": (_i32, [_vp, _i32, _i32]),
    "ocq_batch_get_work": (_i32, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "ocq_batch_autotune": (_i32, [_vp, _i32, _vp]),
    "ocq_batch_set_mode": (_i32, [_vp, _i32]),
    "ocq_batch_set_staging": (_i32, [_vp, _i32]),
    "ocq_batch_get_staging": (_i32, [_vp]),
    "ocq_debug_fail_allocations": (None, [_i32]),
    "ocq_server_snapshot": (_i32, [_vp, _i32, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_i64), _vp]),
    "ocq_server_resume": (_i32, [_vp, ctypes.POINTER(ocq_camera_desc), _vp, _vp, _i64, ctypes.POINTER(_i32)]),
    "ocq_debug_async_bytes_in_use": (_i32, [ctypes.POINTER(ctypes.c_size_t)]),
    "ocq_batch_debug_hold_builds": (_i32, [_vp, _i32]),
    "ocq_build_model_groups": (_i32, [_vp, _i32, _i32, _i32, ocq_region, _i32, _i32, _i32, _vp,
                                      ctypes.POINTER(_vp)]),
    "ocq_redraw": (_i32, [_vp, _i64, _i32, _vp, _vp]),
    "ocq_confusion": (_i32, [_vp, _vp, _i32, _i64, _vp, _vp]),
    "ocq_f_scores": (_i32, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double)]),
    "ocq_batch_get_mode": (_i32, [_vp]),
    "ocq_batch_destroy": (None, [_vp]),
    "ocq_server_create": (_i32, [_sz, _i32, ctypes.POINTER(_vp)]),
    "ocq_server_camera_footprint": (_sz, [ctypes.POINTER(ocq_camera_desc)]),
    "ocq_server_window_bytes": (_sz, [ctypes.POINTER(ocq_camera_desc)]),
    "ocq_server_admit": (_i32, [_vp, ctypes.POINTER(ocq_camera_desc), _vp, ctypes.POINTER(_i32)]),
    "ocq_server_submit": (_i32, [_vp, _i32, _vp, _vp, ctypes.c_uint64]),
    "ocq_server_submit_many": (_i32, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                      ctypes.POINTER(ctypes.c_uint64)]),
    "ocq_server_poll": (_i32, [_vp, ctypes.POINTER(ocq_completion), _i32, ctypes.POINTER(_i32)]),
    "ocq_server_set_batching": (_i32, [_vp, ctypes.c_double, _i32]),
    "ocq_server_release": (_i32, [_vp, _i32]),
    "ocq_server_camera_model": (_i32, [_vp, _i32, ctypes.POINTER(_vp)]),
    "ocq_server_usage": (_i32, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz), ctypes.POINTER(_i64)]),
    "ocq_server_sync": (_i32, [_vp]),
    "ocq_server_destroy": (None, [_vp]),
    "ocq_tune_count": (_i32, [_i32]),
    "ocq_tune_selected": (_i32, [_i32]),
    "ocq_tune_select": (_i32, [_i32, _i32]),
    "ocq_tune_describe": (_i32, [_i32, _i32, ctypes.POINTER(ctypes.c_int32), _i32]),
}

OCQ_TUNE_CLASSIFY_PIXEL, OCQ_TUNE_BUILD_PIXEL, OCQ_TUNE_CLASSIFY_PIXEL_DEEP, OCQ_TUNE_CLASSIFY_BLOCK_DEEP = 0, 1, 2, 3
OCQ_TUNE_CLASSIFY_PIXEL_LIST, OCQ_TUNE_PIXEL_MODEL_FORM, OCQ_TUNE_BUILD_BLOCK = 4, 5, 6
OCQ_BATCH_PERSISTENT, OCQ_BATCH_GRAPH, OCQ_BATCH_GROUPED = 0, 1, 2


def load(path: str | None = None):
    """Load ``libocq.so``.  Raises when it is missing: there is no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or SO
            if not os.path.exists(p):
                raise RuntimeError(f"{p} is missing: build it with __graft_entry__.build() "
                                   "(the octree library has no CPU fallback)")
            lib = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _s(stream):
    if stream is None:
        import torch

        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc: int):
    if rc != OCQ_OK:
        raise OcqError(rc, load().ocq_last_error().decode(errors="replace"))


def _region(kind, block=0):
    if isinstance(kind, ocq_region):
        return kind
    return ocq_region(int(kind), int(block))


class Model:
    """Owns an ``ocq_model*``; freed by ``free()`` or when garbage-collected."""

    def __init__(self, handle: int):
        self.handle = handle

    @property
    def info(self) -> ocq_model_info:
        return ocq_model_get_info(self)

    def free(self):
        if self.handle:
            load().ocq_model_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _h(model):
    return model.handle if isinstance(model, Model) else model


def ocq_status_str(s: int) -> str:
    return load().ocq_status_str(s).decode()


def ocq_last_error() -> str:
    return load().ocq_last_error().decode(errors="replace")


def ocq_version() -> str:
    return load().ocq_version().decode()


def ocq_region_count(H, W, kind, block=0) -> int:
    return int(load().ocq_region_count(H, W, _region(kind, block)))


def ocq_model_footprint(H, W, kind, block, depth) -> int:
    return int(load().ocq_model_footprint(H, W, _region(kind, block), depth))


def ocq_path_code(rgb, npix, depth, codes, stream=None):
    _check(load().ocq_path_code(_p(rgb), npix, depth, _p(codes), _s(stream)))


def ocq_occupancy(frames, n, H, W, kind, block, depth, occ, stream=None):
    _check(load().ocq_occupancy(_p(frames), n, H, W, _region(kind, block), depth, _p(occ), _s(stream)))


def ocq_build_model(frames, N, H, W, kind, block, depth, T, stream=None) -> Model:
    out = ctypes.c_void_p()
    _check(load().ocq_build_model(_p(frames), N, H, W, _region(kind, block), depth, T, _s(stream),
                                  ctypes.byref(out)))
    return Model(out.value)


def ocq_merge_occupancy(occ, parts, N, H, W, kind, block, depth, T, stream=None) -> Model:
    out = ctypes.c_void_p()
    _check(load().ocq_merge_occupancy(_p(occ), parts, N, H, W, _region(kind, block), depth, T, _s(stream),
                                      ctypes.byref(out)))
    return Model(out.value)


def ocq_classify(model, frames, F, mask, stream=None):
    _check(load().ocq_classify(_h(model), _p(frames), F, _p(mask), _s(stream)))


def ocq_build_model_groups(frames, N, H, W, kind, block, depth, T, group, stream=None) -> Model:
    out = ctypes.c_void_p()
    _check(load().ocq_build_model_groups(_p(frames), N, H, W, _region(kind, block), depth, T, group, _s(stream),
                                         ctypes.byref(out)))
    return Model(out.value)


def ocq_redraw(rgb, npix, depth, out, stream=None):
    _check(load().ocq_redraw(_p(rgb), npix, depth, _p(out), _s(stream)))


def ocq_confusion(mask, gt, F, npix, counts, stream=None):
    _check(load().ocq_confusion(_p(mask), _p(gt), F, npix, _p(counts), _s(stream)))


def ocq_f_scores(counts):
    """counts: 4 integers {Tp, Fp, Tn, Fn}; returns (P0, R0, F0, F1)."""
    c = (ctypes.c_uint64 * 4)(*[int(v) for v in counts])
    out = (ctypes.c_double * 4)()
    _check(load().ocq_f_scores(c, out))
    return tuple(out)


def ocq_model_get_info(model) -> ocq_model_info:
    info = ocq_model_info()
    _check(load().ocq_model_get_info(_h(model), ctypes.byref(info)))
    return info


def ocq_model_export(model, dst, words, stream=None):
    _check(load().ocq_model_export(_h(model), _p(dst), words, _s(stream)))


def ocq_model_import(src, info: ocq_model_info, stream=None) -> Model:
    out = ctypes.c_void_p()
    _check(load().ocq_model_import(_p(src), ctypes.byref(info), _s(stream), ctypes.byref(out)))
    return Model(out.value)


def ocq_model_free(model):
    if isinstance(model, Model):
        model.free()
    elif model:
        load().ocq_model_free(model)


def ocq_device_status(stream=None):
    _check(load().ocq_device_status(_s(stream)))


def _hp(x):
    """Host pointer of a numpy array / CPU tensor / integer address."""
    if x is None or isinstance(x, int):
        return x
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    return x.data_ptr()


def ocq_detect_host(train, N, test, F, H, W, kind, block, depth, T, mask, stream=None, keep_model=False):
    """Host buffers in, host masks out (see ocq.h).  Returns the Model when
    ``keep_model``, else None."""
    out = ctypes.c_void_p()
    _check(load().ocq_detect_host(_hp(train), N, _hp(test), F, H, W, _region(kind, block), depth, T, _hp(mask),
                                  _s(stream), ctypes.byref(out) if keep_model else None))
    return Model(out.value) if keep_model else None


def ocq_kernel_launches() -> int:
    return int(load().ocq_kernel_launches())



def ocq_tune_count(kernel: int) -> int:
    return int(load().ocq_tune_count(kernel))


def ocq_tune_selected(kernel: int) -> int:
    return int(load().ocq_tune_selected(kernel))


def ocq_tune_select(kernel: int, variant: int):
    _check(load().ocq_tune_select(kernel, variant))


def ocq_tune_describe(kernel: int, variant: int):
    buf = (ctypes.c_int32 * 5)()
    _check(load().ocq_tune_describe(kernel, variant, buf, 5))
    return list(buf)


def ocq_build_frame_noalloc(frames, N, H, W, depth, T, model, stream=None):
    """Whole-frame model into the caller's device buffer ``model``
    (max(1, 8^depth/64) u64 words, exported layout); allocates nothing.

    The C entry point takes no buffer lengths, so tensors are checked here
    (CUDA, contiguous, large enough) before the call; raw integer addresses
    are passed through unchecked."""
    if not isinstance(frames, int) and frames is not None:
        if not (frames.is_cuda and frames.is_contiguous() and frames.element_size() == 1):
            raise ValueError("frames must be a contiguous CUDA tensor of bytes (uint8)")
        if frames.numel() < N * H * W * 3:
            raise ValueError(f"frames holds {frames.numel()} bytes; N*H*W*3 = {N * H * W * 3} are read")
    if not isinstance(model, int) and model is not None:
        words = max(1, 8 ** depth // 64) if 1 <= depth <= 8 else 1
        if not (model.is_cuda and model.is_contiguous() and model.element_size() == 8):
            raise ValueError("model must be a contiguous CUDA tensor of 8-byte words (int64/uint64)")
        if model.numel() < words:
            raise ValueError(f"model holds {model.numel()} words; depth {depth} writes {words}")
    _check(load().ocq_build_frame_noalloc(_p(frames), N, H, W, depth, T, _p(model), _s(stream)))


class Batch:
    """Owns an ``ocq_batch*`` (many streams, one persistent graph-replayed launch)."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep  # descriptors' buffers must outlive the batch

    def model(self, i: int) -> Model:
        """View of stream i's model (owned by the batch; not freed by the view)."""
        out = ctypes.c_void_p()
        _check(load().ocq_batch_model(self.handle, i, ctypes.byref(out)))
        return _View(out.value)

    def destroy(self):
        if self.handle:
            load().ocq_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class _View(Model):
    def free(self):
        self.handle = None


def ocq_batch_create(descs, stream=None) -> Batch:
    """``descs``: list of dicts with train, N, H, W, kind, block, depth, T, test, F, mask."""
    arr = (ocq_stream_desc * len(descs))()
    for i, d in enumerate(descs):
        arr[i] = ocq_stream_desc(_p(d["train"]), d["N"], d["H"], d["W"], _region(d["kind"], d.get("block", 0)),
                                 d["depth"], d["T"], _p(d.get("test")), d.get("F", 0), _p(d.get("mask")))
    out = ctypes.c_void_p()
    _check(load().ocq_batch_create(arr, len(descs), _s(stream), ctypes.byref(out)))
    return Batch(out.value, descs)


def ocq_batch_run(batch, stream=None):
    _check(load().ocq_batch_run(batch.handle, _s(stream)))


def ocq_batch_status(batch, stream=None):
    _check(load().ocq_batch_status(batch.handle, _s(stream)))


def ocq_batch_model(batch, i) -> Model:
    return batch.model(i)


def ocq_batch_set_work(batch, kind, units):
    _check(load().ocq_batch_set_work(batch.handle, kind, units))


def ocq_batch_get_work(batch, kind):
    u, n = ctypes.c_int(), ctypes.c_int64()
    _check(load().ocq_batch_get_work(batch.handle, kind, ctypes.byref(u), ctypes.byref(n)))
    return u.value, n.value


def ocq_debug_fail_allocations(count):
    load().ocq_debug_fail_allocations(count)


def ocq_debug_async_bytes_in_use() -> int:
    n = ctypes.c_size_t()
    _check(load().ocq_debug_async_bytes_in_use(ctypes.byref(n)))
    return n.value


def ocq_batch_debug_hold_builds(batch, stream):
    _check(load().ocq_batch_debug_hold_builds(batch.handle, stream))


def ocq_batch_set_staging(batch, on):
    _check(load().ocq_batch_set_staging(batch.handle, 1 if on else 0))


def ocq_batch_get_staging(batch) -> int:
    return int(load().ocq_batch_get_staging(batch.handle))


def ocq_batch_set_mode(batch, mode):
    _check(load().ocq_batch_set_mode(batch.handle, mode))


def ocq_batch_get_mode(batch) -> int:
    return int(load().ocq_batch_get_mode(batch.handle))


def ocq_batch_autotune(batch, reps=2, stream=None):
    _check(load().ocq_batch_autotune(batch.handle, reps, _s(stream)))


def ocq_batch_destroy(batch):
    batch.destroy()


class Server:
    """Owns an ``ocq_server*`` (served form)."""

    def __init__(self, handle):
        self.handle = handle

    def destroy(self):
        if self.handle:
            load().ocq_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _camera(H, W, kind, block, depth, T, N, K):
    return ocq_camera_desc(H, W, _region(kind, block), depth, T, N, K)


def ocq_server_create(hbm_budget, max_cameras) -> Server:
    out = ctypes.c_void_p()
    _check(load().ocq_server_create(hbm_budget, max_cameras, ctypes.byref(out)))
    return Server(out.value)


def ocq_server_camera_footprint(H, W, kind, block, depth, T, N, K) -> int:
    d = _camera(H, W, kind, block, depth, T, N, K)
    return int(load().ocq_server_camera_footprint(ctypes.byref(d)))


def ocq_server_window_bytes(H, W, kind, block, depth, T, N, K) -> int:
    d = _camera(H, W, kind, block, depth, T, N, K)
    return int(load().ocq_server_window_bytes(ctypes.byref(d)))


def ocq_server_admit(server, H, W, kind, block, depth, T, N, K, train):
    """Returns the camera id, or None when the server answers OCQ_EBUSY."""
    d = _camera(H, W, kind, block, depth, T, N, K)
    cam = ctypes.c_int()
    rc = load().ocq_server_admit(server.handle, ctypes.byref(d), _p(train), ctypes.byref(cam))
    if rc == OCQ_EBUSY:
        return None
    _check(rc)
    return cam.value


def ocq_server_submit(server, camera, frame, mask, tag=0):
    _check(load().ocq_server_submit(server.handle, camera, _p(frame), _p(mask), tag))


def ocq_server_submit_many(server, cameras, frames, masks, tags):
    """Submits len(cameras) frames at once (continuous batching); frames and
    masks are CUDA tensors or raw device addresses."""
    n = len(cameras)
    if not (len(frames) == len(masks) == len(tags) == n):
        raise ValueError("cameras, frames, masks and tags must have the same length")
    if n == 0:
        return
    cam = (_i32 * n)(*cameras)
    fr = (_vp * n)(*[_p(f) for f in frames])
    mk = (_vp * n)(*[_p(m) for m in masks])
    tg = (ctypes.c_uint64 * n)(*tags)
    _check(load().ocq_server_submit_many(server.handle, n, cam, fr, mk, tg))


def ocq_server_submit_arrays(server, cameras, frame_ptrs, mask_ptrs, tags):
    """ocq_server_submit_many from numpy arrays (int32 cameras, uint64 device
    addresses of frames and masks, uint64 tags), passed without a copy."""
    import numpy as np

    cam = np.ascontiguousarray(cameras, dtype=np.int32)
    fr = np.ascontiguousarray(frame_ptrs, dtype=np.uint64)
    mk = np.ascontiguousarray(mask_ptrs, dtype=np.uint64)
    tg = np.ascontiguousarray(tags, dtype=np.uint64)
    n = cam.shape[0]
    if not (fr.shape[0] == mk.shape[0] == tg.shape[0] == n):
        raise ValueError("cameras, frames, masks and tags must have the same length")
    if n == 0:
        return
    _check(load().ocq_server_submit_many(server.handle, n, cam.ctypes.data_as(ctypes.POINTER(_i32)),
                                         ctypes.cast(fr.ctypes.data, ctypes.POINTER(_vp)),
                                         ctypes.cast(mk.ctypes.data, ctypes.POINTER(_vp)),
                                         tg.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))))


def ocq_server_poll_array(server, max_n=65536):
    """ocq_server_poll into a numpy structured array (fields camera, frame,
    tag, arrival_s, done_s)."""
    import numpy as np

    dt = np.dtype([("camera", np.int32), ("reserved", np.int32), ("frame", np.int64), ("tag", np.uint64),
                   ("arrival_s", np.float64), ("done_s", np.float64)])
    assert dt.itemsize == ctypes.sizeof(ocq_completion)
    buf = np.empty(max_n, dtype=dt)
    n = ctypes.c_int()
    _check(load().ocq_server_poll(server.handle, ctypes.cast(buf.ctypes.data, ctypes.POINTER(ocq_completion)),
                                  max_n, ctypes.byref(n)))
    return buf[:n.value]


def ocq_server_set_batching(server, seconds: float = 0.0, ticks_in_flight: int = 2):
    _check(load().ocq_server_set_batching(server.handle, float(seconds), int(ticks_in_flight)))


def ocq_server_poll(server, max_n=4096):
    buf = (ocq_completion * max_n)()
    n = ctypes.c_int()
    _check(load().ocq_server_poll(server.handle, buf, max_n, ctypes.byref(n)))
    return [(c.camera, c.frame, c.tag, c.arrival_s, c.done_s) for c in buf[:n.value]]


def ocq_server_snapshot(server, camera, model_words, ring_out, stream=None) -> int:
    """Enqueues the camera's checkpoint into ``model_words`` (int64/uint64 CUDA
    tensor) and ``ring_out`` (the window image: at least
    ocq_server_window_bytes bytes; N*H*W*3 always suffices); returns the
    frames submitted."""
    n = ctypes.c_int64()
    _check(load().ocq_server_snapshot(server.handle, camera, _p(model_words), model_words.numel(), _p(ring_out),
                                      ctypes.byref(n), _s(stream)))
    return n.value


def ocq_server_resume(server, H, W, kind, block, depth, T, N, K, model_words, ring, submitted):
    """Returns the camera id, or None when the server answers OCQ_EBUSY."""
    d = _camera(H, W, kind, block, depth, T, N, K)
    cam = ctypes.c_int()
    rc = load().ocq_server_resume(server.handle, ctypes.byref(d), _p(model_words), _p(ring), submitted,
                                  ctypes.byref(cam))
    if rc == OCQ_EBUSY:
        return None
    _check(rc)
    return cam.value


def ocq_server_release(server, camera):
    _check(load().ocq_server_release(server.handle, camera))


def ocq_server_camera_model(server, camera) -> Model:
    out = ctypes.c_void_p()
    _check(load().ocq_server_camera_model(server.handle, camera, ctypes.byref(out)))
    return _View(out.value)


def ocq_server_usage(server):
    u, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_int64()
    _check(load().ocq_server_usage(server.handle, ctypes.byref(u), ctypes.byref(b), ctypes.byref(c)))
    return u.value, b.value, c.value


def ocq_server_sync(server):
    _check(load().ocq_server_sync(server.handle))


def ocq_server_destroy(server):
    server.destroy()
