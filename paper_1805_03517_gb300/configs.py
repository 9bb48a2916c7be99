"""The five matching workloads and their parameters.

Matching parameters follow FlowFields++ (arXiv 1805.03517) where it gives them -- the consistency threshold
eps is 1 px for KITTI-style data and 7 px for Sintel-style data (Table 3) -- and otherwise the readings listed
in the design notes: 8x8 patches with 16 Walsh-Hadamard coefficients per channel, a random-search radius of 2,
3 scales / 4 iterations for the small case and 5 scales / 6 iterations for the rest (the paper itself uses
i = 12 iterations, Sec. 3.1).

Input seeds are 1000 * workload + pair index.
"""
from __future__ import annotations

from dataclasses import dataclass, field

__all__ = ["MatchParams", "PairSpec", "Workload", "WORKLOADS", "TABLE3", "workload"]

HASH_SEED = 0x2018_0503


@dataclass(frozen=True)
class MatchParams:
    n_scales: int = 5
    iters: int = 6
    patch: int = 8
    n_coef: int = 16
    rs_radius: int = 2
    eps: int = 1
    seed: int = HASH_SEED
    rs_radius2: int = 4  # random-search radius of the second inverse field (two-check mode)
    cost: int = 0        # 0: SAD of the WHT descriptors, 1: Hamming distance of 7x7 Census patterns
    sub_scales: int = 0  # 0: none, 1: sub-scales, 2: sub-scales and sub-sub-scales (grids of every 2nd/4th pixel)


@dataclass(frozen=True)
class PairSpec:
    kind: str  # 'rects' | 'kitti' | 'sintel'
    w: int
    h: int
    seed: int
    params: MatchParams

    @property
    def pixels(self) -> int:
        return self.w * self.h


@dataclass(frozen=True)
class Workload:
    name: str
    pairs: tuple = field(default_factory=tuple)
    description: str = ""

    @property
    def pixels(self) -> int:
        return sum(p.pixels for p in self.pairs)


# Table 3: consistency threshold eps (px) and the number of consistent matches s a 3x3 block needs for its
# best match to survive sparsification, per dataset
TABLE3 = {"kitti": {"eps": 1, "min_matches": 7}, "sintel": {"eps": 7, "min_matches": 4}}

SMALL = MatchParams(n_scales=3, iters=4, eps=1)
KITTI = MatchParams(n_scales=5, iters=6, eps=TABLE3["kitti"]["eps"])
SINTEL = MatchParams(n_scales=5, iters=6, eps=TABLE3["sintel"]["eps"])

SERVE_SIZES = ((320, 240, "rects"), (640, 480, "rects"), (1024, 436, "sintel"), (1242, 375, "kitti"))


def _batch48():
    # one parameter set for the whole batch (the KITTI settings, eps = 1, as for the served stream)
    pairs = []
    for i in range(16):
        pairs.append(PairSpec("kitti", 1242, 375, 4000 + i, KITTI))
    for i in range(16):
        pairs.append(PairSpec("sintel", 1024, 436, 4016 + i, KITTI))
    for i in range(16):
        pairs.append(PairSpec("rects", 640, 480, 4032 + i, KITTI))
    return tuple(pairs)


WORKLOADS = {
    "small_128x96": Workload("small_128x96", (PairSpec("rects", 128, 96, 1000, SMALL),),
                             "128x96 value noise, two translated rectangles, L=3, T=4, eps=1"),
    "kitti_1242x375": Workload("kitti_1242x375", (PairSpec("kitti", 1242, 375, 2000, KITTI),),
                               "KITTI-shaped 1242x375 pair, L=5, T=6, eps=1"),
    "sintel_1024x436": Workload("sintel_1024x436", (PairSpec("sintel", 1024, 436, 3000, SINTEL),),
                                "Sintel-shaped 1024x436 pair, L=5, T=6, eps=7"),
    "batch48_mixed": Workload("batch48_mixed", _batch48(),
                              "48 pairs: 16x 1242x375, 16x 1024x436, 16x 640x480, L=5, T=6, eps=1"),
    # the first eight pairs of the batch: a batch whose features (0.95 GB) exceed L2 but that a profiler can
    # replay in a few GB of device memory
    "batch8_kitti_1242x375": Workload("batch8_kitti_1242x375", _batch48()[:8],
                                      "8 KITTI-shaped 1242x375 pairs of the batch, L=5, T=6, eps=1"),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


def serve_sizes(n: int):
    """Sizes (w, h, kind) of the first n pairs of the served stream, uniform over SERVE_SIZES (seeded)."""
    import numpy as np

    rng = np.random.Generator(np.random.PCG64(5000))
    return [SERVE_SIZES[int(c)] for c in rng.integers(0, len(SERVE_SIZES), size=n)]


def serve_pair(i: int) -> PairSpec:
    """The i-th pair of the served stream (one parameter set for the whole stream, eps = 1)."""
    w, h, kind = serve_sizes(i + 1)[i]
    return PairSpec(kind, w, h, 5000 + i, KITTI)
