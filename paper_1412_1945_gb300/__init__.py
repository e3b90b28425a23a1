"""GB300 (sm_103a) octree colour-quantisation background model.

The compute is ``libocq.so`` (CUDA kernels behind the C ABI of
``include/ocq.h``); this package only marshals arguments to it.

``ocq`` holds the same-name bindings of the C entry points; the helpers here
take CUDA tensors of the documented shapes:

* frames: ``uint8[n, H, W, 3]`` (HWC RGB8, contiguous, on the GPU)
* masks: ``uint8[F, H, W]``, 1 = foreground
* exported model: ``uint64[regions, words_per_region]`` (path-code bit order)
"""
from __future__ import annotations

from . import ocq  # noqa: F401
from .ocq import (OCQ_REGION_BLOCK, OCQ_REGION_FRAME, OCQ_REGION_PIXEL, Model, OcqError,  # noqa: F401
                  load)

REGION_KINDS = {"frame": OCQ_REGION_FRAME, "block": OCQ_REGION_BLOCK, "pixel": OCQ_REGION_PIXEL}


def _kind(kind):
    return REGION_KINDS[kind] if isinstance(kind, str) else int(kind)


def _frames(t, name="frames"):
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.uint8 and t.dim() == 4
            and t.shape[3] == 3 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA uint8 tensor [n, H, W, 3]")
    return t


def build_model(frames, depth: int, T: int, kind="pixel", block: int = 0, stream=None) -> Model:
    """S1-S3: merged model of the training frames ``frames`` [N, H, W, 3]."""
    _frames(frames)
    N, H, W, _ = frames.shape
    return ocq.ocq_build_model(frames, N, H, W, _kind(kind), block, depth, T, stream)


def classify(model: Model, frames, mask=None, stream=None):
    """S4: foreground mask [F, H, W] of ``frames`` [F, H, W, 3]."""
    import torch

    _frames(frames)
    F, H, W, _ = frames.shape
    if mask is None:
        mask = torch.empty((F, H, W), dtype=torch.uint8, device=frames.device)
    ocq.ocq_classify(model, frames, F, mask, stream)
    return mask


def export_model(model: Model, stream=None):
    """The model as uint64[regions, words_per_region] on the GPU (path-code bit order)."""
    import torch

    info = model.info
    out = torch.empty((info.regions, info.words_per_region), dtype=torch.int64, device="cuda")
    ocq.ocq_model_export(model, out, out.numel(), stream)
    return out


def import_model(words, H, W, kind, block, depth, T=1, N=1, stream=None) -> Model:
    info = ocq.ocq_model_info(H=H, W=W, region_kind=_kind(kind), block=block, depth=depth, T=T, N=N)
    return ocq.ocq_model_import(words, info, stream)


def path_code(rgb, depth: int, stream=None):
    """S1 alone: uint32 path codes of ``rgb`` (CUDA uint8 tensor, last dim 3)."""
    import torch

    n = rgb.numel() // 3
    out = torch.empty(n, dtype=torch.int32, device=rgb.device)
    ocq.ocq_path_code(rgb, n, depth, out, stream)
    return out


def occupancy(frames, depth: int, kind="frame", block: int = 0, stream=None):
    """S2 alone: per-frame, per-region leaf bitsets [n, regions, words_per_region]."""
    import torch

    _frames(frames)
    n, H, W, _ = frames.shape
    R = ocq.ocq_region_count(H, W, _kind(kind), block)
    wpr = 1 if depth <= 2 else 1 << (3 * depth - 6)
    out = torch.empty((n, R, wpr), dtype=torch.int64, device=frames.device)
    ocq.ocq_occupancy(frames, n, H, W, _kind(kind), block, depth, out, stream)
    return out


def device_status(stream=None):
    """Synchronise and raise OcqError(OCQ_ETIMEOUT) if a bounded device wait gave up."""
    ocq.ocq_device_status(stream)


def build_model_groups(frames, depth: int, T: int, group: int, kind="pixel", block: int = 0, stream=None) -> Model:
    """S1-S3 with one tree per group of ``group`` consecutive frames; T counts trees."""
    _frames(frames)
    N, H, W, _ = frames.shape
    return ocq.ocq_build_model_groups(frames, N, H, W, _kind(kind), block, depth, T, group, stream)


def redraw(rgb, depth: int, out=None, stream=None):
    """Each colour of ``rgb`` (CUDA uint8, last dim 3) as its leaf colour at ``depth``."""
    import torch

    if out is None:
        out = torch.empty_like(rgb)
    ocq.ocq_redraw(rgb, rgb.numel() // 3, depth, out, stream)
    return out


def confusion(mask, gt, stream=None):
    """Per frame {Tp, Fp, Tn, Fn} of ``mask`` against ``gt`` (CUDA uint8 [F, ...]) as int64 [F, 4]."""
    import torch

    F = mask.shape[0]
    counts = torch.empty((F, 4), dtype=torch.int64, device=mask.device)
    ocq.ocq_confusion(mask, gt, F, mask[0].numel() if F else 0, counts, stream)
    return counts


def f_scores(counts):
    """P0, R0, F0 (the paper's Sec. 5 scores) and foreground F1 from counts {Tp, Fp, Tn, Fn}."""
    p0, r0, f0, f1 = ocq.ocq_f_scores(counts)
    return {"P0": p0, "R0": r0, "F0": f0, "F1": f1}
