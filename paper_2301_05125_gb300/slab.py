"""Probe-slab split of one volume's update over several ranks (one GPU each).

The update's work is per probe except for three places where a probe needs
other probes' data, and those fix the exchange steps of a frame:

  1. W_p sums the octant sums G (of the trigger Tr) over the 5x5x5 probes
     around p (Sec. 4.1, spatial convolution): a rank needs G of the two
     z-planes on each side of its slab -> halo exchange of G;
  2. the allocation spreads one fixed budget over all probes (Sec. 3.4):
     every rank needs every W_p -> all-gather of W, after which each rank
     computes the same integer allocation (no reduction order to agree on);
  3. the shading of a ray reads the previous frame's atlases at its hit
     point, and rays have no length limit, so a hit can fall in any cage of
     the volume -> all-gather of the tiles each rank blended.

A rank owns whole z-planes [z0, z1), i.e. the contiguous probes
[z0 X Y, z1 X Y).  Per frame: step 0 (pilot rays and the change state of its
probes), halo G; step 1 (W of its probes), gather W; step 2 (allocation,
adaptive rays and blend of its probes), gather the tiles.  Each rank's probes
then end exactly as an unsplit update leaves them.

The data movement is host-driven between the steps, so no kernel waits on
another rank.  `DistExchange` moves the slices with torch.distributed
(NCCL for device tensors, gloo for host tensors); `LocalExchange` moves
them between several ranks' volumes held by one process.  A backend gives
the steps and the slices of its per-probe arrays: `CudaSlabRank` wraps a
volume of the C library (adgi_update_slab / adgi_slab_copy).
"""
from dataclasses import dataclass
from typing import List, Sequence, Tuple

HALO_PLANES = 2  # the 5x5x5 stencil reaches two planes beyond the slab


def slab_ranges(dims: Sequence[int], n_ranks: int) -> List[Tuple[int, int]]:
    """Probe range [p0, p1) of each rank: the z-planes split as evenly as
    possible (the first Z mod n ranks take one plane more)."""
    X, Y, Z = (int(d) for d in dims)
    if n_ranks < 1 or n_ranks > Z:
        raise ValueError("need 1 <= ranks <= %d z-planes" % Z)
    out, z = [], 0
    for r in range(n_ranks):
        nz = Z // n_ranks + (1 if r < Z % n_ranks else 0)
        out.append((z * X * Y, (z + nz) * X * Y))
        z += nz
    return out


def halo_ranges(dims: Sequence[int], rng: Tuple[int, int], width: int = HALO_PLANES) -> List[Tuple[int, int]]:
    """The probes within `width` z-planes below and above slab rng (clipped to
    the grid), as up to two ranges."""
    X, Y, Z = (int(d) for d in dims)
    plane = X * Y
    z0, z1 = rng[0] // plane, rng[1] // plane
    out = []
    if z0 > 0:
        out.append((max(z0 - width, 0) * plane, z0 * plane))
    if z1 < Z:
        out.append((z1 * plane, min(z1 + width, Z) * plane))
    return out


def _overlap(a, b):
    lo, hi = max(a[0], b[0]), min(a[1], b[1])
    return (lo, hi) if lo < hi else None


@dataclass
class SlabPart:
    """One rank's share: its backend and its probe range."""
    backend: object
    rank: int
    rng: Tuple[int, int]


class LocalExchange:
    """All ranks' volumes in one process: slices are copied directly."""

    def __init__(self, dims, ranges):
        self.dims, self.ranges = dims, ranges

    def halo(self, parts, which):
        for d in parts:
            for s in parts:
                if s is d:
                    continue
                for h in halo_ranges(self.dims, d.rng):
                    ov = _overlap(h, s.rng)
                    if ov:
                        d.backend.put(which, ov[0], ov[1], s.backend.get(which, ov[0], ov[1]))

    def gather(self, parts, which):
        for s in parts:
            data = s.backend.get(which, *s.rng)
            for d in parts:
                if d is not s:
                    d.backend.put(which, s.rng[0], s.rng[1], data)


class DistExchange:
    """One rank per process: slices move with torch.distributed (point to
    point for the halo, one broadcast per owner for the gathers, which also
    handles slabs of unequal size)."""

    def __init__(self, dims, ranges, group=None):
        import torch.distributed as dist

        self.dist, self.group = dist, group
        self.dims, self.ranges = dims, ranges
        self.me = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        if self.world != len(ranges):
            raise ValueError("one probe range per rank")

    def halo(self, parts, which):
        (mine,) = parts
        dist = self.dist
        ops, recv = [], []
        for s in range(self.world):  # what this rank needs from rank s
            if s == self.me:
                continue
            for h in halo_ranges(self.dims, self.ranges[self.me]):
                ov = _overlap(h, self.ranges[s])
                if ov:
                    buf = mine.backend.empty(which, ov[0], ov[1])
                    recv.append((ov, buf))
                    ops.append(dist.irecv(buf, src=s, group=self.group))
        for d in range(self.world):  # what rank d needs from this rank
            if d == self.me:
                continue
            for h in halo_ranges(self.dims, self.ranges[d]):
                ov = _overlap(h, self.ranges[self.me])
                if ov:
                    ops.append(dist.isend(mine.backend.get(which, ov[0], ov[1]), dst=d, group=self.group))
        for op in ops:
            op.wait()
        for ov, buf in recv:
            mine.backend.put(which, ov[0], ov[1], buf)

    def gather(self, parts, which):
        (mine,) = parts
        for r in range(self.world):
            lo, hi = self.ranges[r]
            if hi <= lo:
                continue
            buf = mine.backend.get(which, lo, hi) if r == self.me else mine.backend.empty(which, lo, hi)
            self.dist.broadcast(buf, src=r, group=self.group)
            if r != self.me:
                mine.backend.put(which, lo, hi, buf)


def slab_update(parts: List[SlabPart], exchange, frame) -> None:
    """One frame of the split update for the ranks held by this process
    (one with DistExchange, all of them with LocalExchange).  `frame` is
    passed to the backends as they expect it."""
    for p in parts:
        p.backend.step(0, frame, *p.rng)
    for which in parts[0].backend.HALO:
        exchange.halo(parts, which)
    for p in parts:
        p.backend.step(1, frame, *p.rng)
    exchange.gather(parts, "W")
    for p in parts:
        p.backend.step(2, frame, *p.rng)
    for which in parts[0].backend.ATLAS:
        exchange.gather(parts, which)


class CudaSlabRank:
    """Backend over a volume of the C library.  The slices are device
    tensors of raw bytes; the volume must run on the stream torch uses for
    the collectives (torch.cuda.current_stream() of its device), so the
    copies and the collectives are ordered."""

    HALO = ("G",)
    ATLAS = ("IRR", "DEP", "DEP_N")

    def __init__(self, volume, device):
        from . import adgi

        self.adgi, self.vol, self.device = adgi, volume, device

    def step(self, k, frame, p0, p1):
        self.adgi.adgi_update_slab(self.vol.h, frame, k, p0, p1)

    def empty(self, which, p0, p1):
        import torch

        return torch.empty(self.adgi.adgi_slab_bytes(self.vol.h, which, p0, p1), dtype=torch.uint8,
                           device=self.device)

    def get(self, which, p0, p1):
        buf = self.empty(which, p0, p1)
        if buf.numel():
            self.adgi.adgi_slab_copy(self.vol.h, which, p0, p1, buf, 0)
        return buf

    def put(self, which, p0, p1, buf):
        if buf.numel():
            self.adgi.adgi_slab_copy(self.vol.h, which, p0, p1, buf, 1)
