"""x-slab decomposition of one capillary over several lattices (halo exchange).

The paper's Introduction notes that the lattice Boltzmann method parallelises
naturally: every node needs only its neighbours.  A run of nx columns is cut
into slabs of owned columns [x_p, x_{p+1}); slab p is advanced as a lattice of
w_p + 4 columns whose local column c holds global column (x_p - 2 + c) mod nx.
Columns 0, 1 and w_p + 2, w_p + 3 are halos: after every step they are
overwritten with the neighbours' edge columns (their populations after that
step), through lbm_set_columns.  The pull of an owned column reaches one
column and the densities of its force one more (Eqs. 2, 9), so every owned
column gets exactly the inputs it has in the undivided lattice, and the slabs
together reproduce the undivided run bit for bit.  Only populations travel:
36 values per halo node and step.

Geometry: each slab gets the columns of the run's solid mask (the plates
become a mask), and no front tracking (fronts are a property of the whole
capillary).  Exchange: `exchange_local` for slabs held by one process,
`SlabRank` for one slab per rank over torch.distributed point-to-point
send/recv (NCCL between GPUs, gloo between CPU processes).
"""
from __future__ import annotations

import numpy as np

HALO = 2   # columns of halo on each side


def slab_bounds(nx: int, parts: int):
    """Owned column ranges [(x0, x1), ...] of `parts` slabs of near-equal width."""
    if parts < 1 or nx < 4 * parts:
        raise ValueError("each slab needs at least 4 owned columns")
    base, extra = divmod(nx, parts)
    out, x = [], 0
    for p in range(parts):
        w = base + (1 if p < extra else 0)
        out.append((x, x + w))
        x += w
    return out


def solid_mask(geom: dict) -> np.ndarray:
    """[ny][nx] uint8 solid flags of a geometry: its mask, or the plates
    (rows y_bot and y_top over columns [cap_x0, cap_x1))."""
    if geom.get("mask") is not None:
        return np.ascontiguousarray(geom["mask"], dtype=np.uint8)
    m = np.zeros((geom["ny"], geom["nx"]), np.uint8)
    for y in (geom["y_bot"], geom["y_top"]):
        if y >= 0:
            m[y, geom["cap_x0"]:geom["cap_x1"]] = 1
    return m


def _columns(a: np.ndarray, x0: int, x1: int) -> np.ndarray:
    """Columns x0 - HALO .. x1 + HALO - 1 of a [.., nx] array, periodic in x."""
    nx = a.shape[-1]
    return np.ascontiguousarray(np.take(a, np.arange(x0 - HALO, x1 + HALO) % nx, axis=-1))


def slab_run(run: dict, x0: int, x1: int, nA: np.ndarray, nB: np.ndarray) -> dict:
    """The lattice description of the slab owning columns [x0, x1) of `run`
    (initial fields nA, nB of the whole run, [ny][nx])."""
    g = run["geom"]
    geom = dict(nx=x1 - x0 + 2 * HALO, ny=g["ny"], cap_x0=0, cap_x1=0, y_bot=-1, y_top=-1,
                mask=_columns(solid_mask(g), x0, x1))
    return dict(geom=geom, params=dict(run["params"]), init=("fields", _columns(nA, x0, x1), _columns(nB, x0, x1)))


class Slab:
    """One slab: a lattice of w + 4 columns (made by `factory(run_dict)`,
    by default the GPU Lattice) and its owned range [x0, x1)."""

    def __init__(self, run: dict, x0: int, x1: int, nA: np.ndarray, nB: np.ndarray, factory=None, **lattice_kw):
        self.x0, self.x1, self.w = x0, x1, x1 - x0
        local = slab_run(run, x0, x1, nA, nB)
        if factory is None:
            from .lbm import Lattice
            factory = lambda r: Lattice(r, **lattice_kw)   # noqa: E731
        self.lat = factory(local)

    def step(self) -> None:
        self.lat.step(1)

    def left_edge(self):
        return self.lat.get_columns(HALO, HALO)                # owned columns x0, x0 + 1

    def right_edge(self):
        return self.lat.get_columns(self.w, HALO)              # owned columns x1 - 2, x1 - 1

    def set_halos(self, from_left, from_right) -> None:
        self.lat.set_columns(0, from_left)                     # columns x0 - 2, x0 - 1
        self.lat.set_columns(self.w + HALO, from_right)        # columns x1, x1 + 1

    def owned(self, field: np.ndarray) -> np.ndarray:
        """The owned columns of a local [.., w + 4] array."""
        return field[..., HALO:HALO + self.w]


def exchange_local(slabs) -> None:
    """Halo exchange among slabs of one process, in ring order (periodic x):
    every slab's edges are read before any halo is written."""
    edges = [(s.left_edge(), s.right_edge()) for s in slabs]
    P = len(slabs)
    for p, s in enumerate(slabs):
        s.set_halos(edges[(p - 1) % P][1], edges[(p + 1) % P][0])


def step_local(slabs, n: int) -> None:
    """n steps of the decomposed run held by one process."""
    for _ in range(n):
        for s in slabs:
            s.step()
        exchange_local(slabs)


class SlabRank:
    """The slab of this rank of a torch.distributed group: rank r owns slab r
    of slab_bounds(nx, world) and exchanges its edges with ranks r - 1 and
    r + 1 (periodic) by point-to-point send/recv after every step.  The
    tensors live where the lattice keeps them (CUDA for the GPU lattice, so
    NCCL moves them between GPUs; CPU under gloo)."""

    def __init__(self, run: dict, nA: np.ndarray, nB: np.ndarray, group=None, factory=None, **lattice_kw):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        x0, x1 = slab_bounds(run["geom"]["nx"], self.world)[self.rank]
        self.slab = Slab(run, x0, x1, nA, nB, factory=factory, **lattice_kw)

    def step(self, n: int = 1) -> None:
        for _ in range(n):
            self.slab.step()
            self.exchange()

    def exchange(self) -> None:
        dist, s = self.dist, self.slab
        left, right = s.left_edge(), s.right_edge()
        if self.world == 1:
            s.set_halos(right, left)
            return
        from_left, from_right = left.clone(), right.clone()
        g = self.group
        glob = (lambda r: dist.get_global_rank(g, r)) if g is not None else (lambda r: r)
        prev, nxt = glob((self.rank - 1) % self.world), glob((self.rank + 1) % self.world)
        # tag 0 carries a right edge to the next rank, tag 1 a left edge to the previous one
        ops = [dist.P2POp(dist.isend, right, nxt, g, 0), dist.P2POp(dist.isend, left, prev, g, 1),
               dist.P2POp(dist.irecv, from_left, prev, g, 0), dist.P2POp(dist.irecv, from_right, nxt, g, 1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        s.set_halos(from_left, from_right)
