"""Placement of whole scenes on devices (one process per GPU).

Independent scenes -- the batched Newton step and the served request
stream -- shard across GPUs with no exchange on the data path: each device
owns whole scenes, steps them with its own context, and only host-side
bookkeeping (which scene went where, per-rank timings and results) is
gathered. These functions are pure host logic, the same on every rank, so
every rank computes the same placement without communicating.
"""
from __future__ import annotations

import heapq
from typing import Dict, List, Sequence


def place_by_footprint(footprints: Sequence[int], n_devices: int) -> List[int]:
    """Device of each scene: largest footprint first, each to the device
    with the smallest total so far (ties: the lower device index). Balances
    device memory and, since work grows with size, device time."""
    if n_devices < 1:
        raise ValueError("n_devices must be >= 1")
    order = sorted(range(len(footprints)), key=lambda i: (-int(footprints[i]), i))
    heap = [(0, d) for d in range(n_devices)]
    heapq.heapify(heap)
    dev = [0] * len(footprints)
    for i in order:
        load, d = heapq.heappop(heap)
        dev[i] = d
        heapq.heappush(heap, (load + int(footprints[i]), d))
    return dev


def route_stream(footprints: Sequence[int], n_devices: int) -> List[int]:
    """Device of each request of an arrival-ordered stream: each request
    goes, in arrival order, to the device with the least footprint routed so
    far (a request cannot wait for later ones to be known)."""
    if n_devices < 1:
        raise ValueError("n_devices must be >= 1")
    load = [0] * n_devices
    dev = []
    for f in footprints:
        d = min(range(n_devices), key=lambda j: (load[j], j))
        dev.append(d)
        load[d] += int(f)
    return dev


def mine(placement: Sequence[int], rank: int) -> List[int]:
    """Indices of the scenes placed on `rank`, in their original order."""
    return [i for i, d in enumerate(placement) if d == rank]


def merge(parts: Sequence[Dict[int, object]], n: int) -> List[object]:
    """Per-rank {scene index: result} dictionaries -> results in scene order;
    every scene must appear exactly once."""
    out: List[object] = [None] * n
    seen = [False] * n
    for p in parts:
        for i, v in p.items():
            if seen[i]:
                raise ValueError("scene %d placed twice" % i)
            seen[i] = True
            out[i] = v
    if not all(seen):
        raise ValueError("scene %d not placed" % seen.index(False))
    return out
