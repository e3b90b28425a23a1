"""Seeded synthetic inputs for the octree background model.

This package is the one module that both the oracle (test infrastructure) and
the CUDA path consume.  It holds input generation only -- scene tables,
per-pixel content, workload presets -- and none of the method's arithmetic.

* ``make_scene`` builds a scene blob (``scene.py``).
* ``fill_host`` renders frames on the CPU (gcc-built ``libocq_synth_host.so``).
* ``fill_device`` renders the same bytes on the GPU (nvcc-built
  ``libocq_synth_dev.so``), so full-size workloads never cross PCIe/C2C.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .scene import make_scene, scene_hw  # noqa: F401
from . import configs  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_HOST_SO = os.path.join(_HERE, "libocq_synth_host.so")
_DEV_SO = os.path.join(_HERE, "libocq_synth_dev.so")
_lock = threading.Lock()
_host_lib = None
_dev_lib = None


def _stale(target: str, sources) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def build_commands(nvcc: str = "nvcc"):
    """(target, command) pairs that compile the two generator libraries."""
    hdr = os.path.join(_CSRC, "synth_pixel.h")
    host_src = os.path.join(_CSRC, "synth_host.c")
    dev_src = os.path.join(_CSRC, "synth_dev.cu")
    cmds = []
    if _stale(_HOST_SO, [hdr, host_src]):
        cmds.append((_HOST_SO, ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", _HOST_SO, host_src]))
    if _stale(_DEV_SO, [hdr, dev_src]):
        cmds.append((_DEV_SO, [nvcc, "-O3", "-gencode", "arch=compute_103a,code=sm_103a",
                               "-Xcompiler", "-fPIC", "-shared", "-o", _DEV_SO, dev_src]))
    return cmds


def build(device: bool = True) -> None:
    """Compile the generator libraries in-tree (host: gcc; device: nvcc sm_103a)."""
    cmds = build_commands()
    if not device:
        cmds = [c for c in cmds if c[0] != _DEV_SO]
    procs = [(t, subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)) for t, c in cmds]
    for t, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"building {t} failed:\n{out.decode(errors='replace')}")


def _load_host():
    global _host_lib
    with _lock:
        if _host_lib is None:
            if _stale(_HOST_SO, [os.path.join(_CSRC, "synth_pixel.h"), os.path.join(_CSRC, "synth_host.c")]):
                build(device=False)
            lib = ctypes.CDLL(_HOST_SO)
            lib.ocq_synth_fill_host.restype = ctypes.c_int
            lib.ocq_synth_fill_host.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                ctypes.c_void_p, ctypes.c_void_p]
            lib.ocq_synth_fill_pixels_host.restype = ctypes.c_int
            lib.ocq_synth_fill_pixels_host.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                                       ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
            _host_lib = lib
    return _host_lib


def _load_dev():
    global _dev_lib
    with _lock:
        if _dev_lib is None:
            if not os.path.exists(_DEV_SO):
                raise RuntimeError("libocq_synth_dev.so is not built; run __graft_entry__.build()")
            lib = ctypes.CDLL(_DEV_SO)
            lib.ocq_synth_fill_device.restype = ctypes.c_int
            lib.ocq_synth_fill_device.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                                                  ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p]
            _dev_lib = lib
    return _dev_lib


def fill_host(scene: np.ndarray, frame0: int, nframes: int, with_gt: bool = False):
    """Render frames [frame0, frame0+nframes) on the CPU.

    Returns ``rgb`` as ``uint8[nframes, H, W, 3]`` (and ``gt`` as
    ``uint8[nframes, H, W]``, 1 = foreground object, when ``with_gt``)."""
    lib = _load_host()
    scene = np.ascontiguousarray(scene, dtype=np.int32)
    H, W = scene_hw(scene)
    rgb = np.empty((nframes, H, W, 3), dtype=np.uint8)
    gt = np.empty((nframes, H, W), dtype=np.uint8) if with_gt else None
    rc = lib.ocq_synth_fill_host(scene.ctypes.data, frame0, nframes, rgb.ctypes.data,
                                 gt.ctypes.data if gt is not None else None)
    if rc != 0:
        raise RuntimeError("ocq_synth_fill_host failed")
    return (rgb, gt) if with_gt else rgb


def fill_pixels_host(scene: np.ndarray, frame0: int, nframes: int, idx) -> np.ndarray:
    """Render only the pixel locations ``idx`` (row-major indices) of frames
    [frame0, frame0+nframes): returns ``uint8[nframes, 1, len(idx), 3]``, a
    1-row frame that per-pixel regions treat exactly like the full frame."""
    lib = _load_host()
    scene = np.ascontiguousarray(scene, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty((nframes, 1, idx.size, 3), dtype=np.uint8)
    if lib.ocq_synth_fill_pixels_host(scene.ctypes.data, frame0, nframes, idx.ctypes.data, idx.size,
                                      out.ctypes.data) != 0:
        raise RuntimeError("ocq_synth_fill_pixels_host failed")
    return out


def fill_device(scene: np.ndarray, frame0: int, nframes: int, out, gt=None, stream=None):
    """Render frames [frame0, frame0+nframes) into the CUDA tensor ``out``
    (``uint8``, ``nframes*H*W*3`` elements, contiguous) and optionally ``gt``."""
    import torch

    lib = _load_dev()
    H, W = scene_hw(scene)
    need = nframes * H * W * 3
    if not out.is_cuda or out.dtype != torch.uint8 or not out.is_contiguous() or out.numel() < need:
        raise ValueError("out must be a contiguous CUDA uint8 tensor large enough for the frames")
    sc = torch.from_numpy(np.ascontiguousarray(scene, dtype=np.int32)).to(out.device)
    st = stream if stream is not None else torch.cuda.current_stream(out.device)
    rc = lib.ocq_synth_fill_device(sc.data_ptr(), H, W, frame0, nframes, out.data_ptr(),
                                   gt.data_ptr() if gt is not None else None, st.cuda_stream)
    if rc != 0:
        raise RuntimeError(f"ocq_synth_fill_device failed: cudaError {rc}")
    st.synchronize()
    del sc
