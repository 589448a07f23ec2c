"""Rank geometry and halo-exchange data plane of the domain decomposition
(Sections 2.1 and 2.2 and Algorithm 3 of the thesis) for ranks that are
processes.

The virtual ranks of one GPU (``Decomposition``, the ``dd_decomp_*`` calls of
the C ABI) move their face messages with device copies inside the library.
Ranks that are processes exchange the same messages through
``torch.distributed``: ``HaloPlan`` gives a rank of a process grid its local
lattice, its offset, its neighbours and the order of the sites on each face;
``exchange`` posts one send and one receive per split direction and message
kind, over whatever backend the process group has (gloo for host tensors,
NCCL for device tensors).  Message kinds follow Algorithm 3:

* ``LAMBDA`` (kind 0): the projected spinors of the rank's lowest mu slice
  (its inner boundary), sent in the negative mu direction;
* ``CHI`` (kind 1): the projected spinors of its highest mu slice times
  U_mu^H, sent in the positive mu direction.

Faces list their sites by the three other local coordinates, lexicographic in
the order T, Z, Y, X, the order the library's face buffers use.  Nothing here
does arithmetic on field values.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

LAMBDA, CHI = 0, 1


def rank_coords(rank: int, grid) -> tuple:
    """Grid coordinates (T, Z, Y, X; X fastest) of a rank."""
    c = []
    for g in reversed(tuple(grid)):
        c.append(rank % g)
        rank //= g
    return tuple(reversed(c))


def rank_of(coords, grid) -> int:
    r = 0
    for c, g in zip(coords, grid):
        r = r * g + (c % g)
    return r


@dataclass(frozen=True)
class HaloPlan:
    dims: tuple      # global extents (nT, nZ, nY, nX)
    grid: tuple      # ranks per direction
    rank: int

    def __post_init__(self):
        for n, g in zip(self.dims, self.grid):
            if g < 1 or n % g or (n // g) % 2:
                raise ValueError(f"extent {n} does not split into {g} even local extents")

    @property
    def coords(self):
        return rank_coords(self.rank, self.grid)

    @property
    def local(self):
        return tuple(n // g for n, g in zip(self.dims, self.grid))

    @property
    def offset(self):
        return tuple(c * l for c, l in zip(self.coords, self.local))

    @property
    def nranks(self):
        return int(np.prod(self.grid))

    def split(self, mu: int) -> bool:
        """Whether direction mu crosses ranks (its seams are exchanged)."""
        return self.grid[mu] > 1

    def neighbour(self, mu: int, step: int) -> int:
        c = list(self.coords)
        c[mu] += step
        return rank_of(c, self.grid)

    def local_sites(self) -> np.ndarray:
        """Global lexicographic indices of the rank's sites, in local
        lexicographic order."""
        t, z, y, x = np.meshgrid(*[np.arange(o, o + n) for o, n in zip(self.offset, self.local)], indexing="ij")
        nT, nZ, nY, nX = self.dims
        return (((t * nZ + z) * nY + y) * nX + x).reshape(-1)

    def face_sites(self, mu: int, side: int) -> np.ndarray:
        """Local lexicographic indices of the sites of the lowest (side 0) or
        highest (side 1) mu slice, in face order."""
        n = self.local
        ranges = [np.arange(k) for k in n]
        ranges[mu] = np.array([0 if side == 0 else n[mu] - 1])
        t, z, y, x = np.meshgrid(*ranges, indexing="ij")
        return (((t * n[1] + z) * n[2] + y) * n[3] + x).reshape(-1)

    def face_size(self, mu: int) -> int:
        return int(np.prod([k for d, k in enumerate(self.local) if d != mu]))

    def messages(self):
        """(mu, kind, destination rank, source rank) of every message this rank
        sends and receives in one exchange round."""
        out = []
        for mu in range(4):
            if not self.split(mu):
                continue
            out.append((mu, LAMBDA, self.neighbour(mu, -1), self.neighbour(mu, +1)))
            out.append((mu, CHI, self.neighbour(mu, +1), self.neighbour(mu, -1)))
        return out


def tag(mu: int, kind: int) -> int:
    return 2 * mu + kind


def exchange(plan: HaloPlan, sends: dict, recvs: dict, group=None) -> None:
    """Send sends[(mu, kind)] to its destination and receive recvs[(mu, kind)]
    (preallocated, same shape) from its source, for every message of the
    plan; returns when all have completed.  For grid[mu] = 2 both neighbours
    are the same rank: the tags keep the two kinds apart."""
    import torch.distributed as dist
    reqs = []
    for mu, kind, dst, src in plan.messages():
        reqs.append(dist.irecv(recvs[(mu, kind)], src=src, group=group, tag=tag(mu, kind)))
    for mu, kind, dst, src in plan.messages():
        reqs.append(dist.isend(sends[(mu, kind)], dst=dst, group=group, tag=tag(mu, kind)))
    for r in reqs:
        r.wait()
