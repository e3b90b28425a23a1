"""Named workload presets (parameters only; no method arithmetic).

Region kinds use the library's numbering: 0 whole frame, 1 b x b blocks,
2 single pixel locations.  Seeds are ``0x14121945 + k`` for preset k.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from .scene import TableRng

REGION_FRAME, REGION_BLOCK, REGION_PIXEL = 0, 1, 2
SEED_BASE = 0x14121945


@dataclass(frozen=True)
class Workload:
    name: str
    scene_kind: str
    H: int
    W: int
    N: int            # training frames
    F: int            # test frames
    region: int
    block: int
    depth: int
    T: int
    seed: int
    stream: int = 0


TINY_FRAME = Workload("tiny_frame_160x120_d4", "clusters", 120, 160, 8, 8, REGION_FRAME, 0, 4, 4, SEED_BASE + 0)
BLOCKS_320x240 = Workload("blocks16_320x240_d5", "sway", 240, 320, 30, 300, REGION_BLOCK, 16, 5, 15, SEED_BASE + 1)
PIXEL_1080P = Workload("pixel_1920x1080_d3", "bimodal", 1080, 1920, 50, 1000, REGION_PIXEL, 0, 3, 10, SEED_BASE + 2)

PRESETS = {w.name: w for w in (TINY_FRAME, BLOCKS_320x240, PIXEL_1080P)}

BATCH_RESOLUTIONS = ((320, 240), (640, 480), (1280, 720), (1920, 1080))
SERVE_RESOLUTIONS = BATCH_RESOLUTIONS + ((3840, 2160),)


def batched_streams(n_streams: int = 64, test_frames: int = 100, seed: int = SEED_BASE + 3):
    """Uneven camera streams: resolution uniform over 320x240..1920x1080,
    depth 3-5, region 1x1 / 8x8 / whole frame, N in [20, 50], T = ceil(N/3),
    content cluster- or sway-style by a coin."""
    rng = TableRng(seed, 0, 200)
    out = []
    for s in range(n_streams):
        W, H = BATCH_RESOLUTIONS[rng.randint(0, 3)]
        depth = rng.randint(3, 5)
        rk = rng.randint(0, 2)
        region, block = ((REGION_PIXEL, 0), (REGION_BLOCK, 8), (REGION_FRAME, 0))[rk]
        N = rng.randint(20, 50)
        T = math.ceil(N / 3)
        kind = "clusters" if rng.randint(0, 1) == 0 else "sway"
        out.append(Workload(f"stream{s}", kind, H, W, N, test_frames, region, block, depth, T, seed, s))
    return out


@dataclass
class ServeStream:
    wl: Workload
    join_s: float
    fps: float = 30.0
    n_frames: int = 0
    arrivals: list = field(default_factory=list)


def serving_streams(n_streams: int = 256, frames_per_stream: int = 90, join_rate: float = 25.6,
                    fps: float = 30.0, window: int = 30, seed: int = SEED_BASE + 4):
    """Camera streams joining as a Poisson process (``join_rate`` per second),
    each then sending frames as a Poisson process at ``fps``; resolutions up to
    3840x2160, depth 3-5, N = ``window`` training frames, T = 10, region mix as
    in ``batched_streams``."""
    rng = TableRng(seed, 0, 300)

    def expo(rate):
        u = (rng.u64() >> 11) * (1.0 / (1 << 53))
        return -math.log(1.0 - u) / rate

    out = []
    t = 0.0
    for s in range(n_streams):
        t += expo(join_rate)
        W, H = SERVE_RESOLUTIONS[rng.randint(0, 4)]
        depth = rng.randint(3, 5)
        rk = rng.randint(0, 2)
        region, block = ((REGION_PIXEL, 0), (REGION_BLOCK, 8), (REGION_FRAME, 0))[rk]
        kind = "clusters" if rng.randint(0, 1) == 0 else "sway"
        wl = Workload(f"cam{s}", kind, H, W, window, frames_per_stream, region, block, depth, 10, seed, s)
        st = ServeStream(wl, t, fps, frames_per_stream)
        a = t
        for _ in range(frames_per_stream):
            a += expo(fps)
            st.arrivals.append(a)
        out.append(st)
    return out
