"""Split-domain runs: one tile of a checkerboard per process (Secs. 4-5 of
the paper), the tiles exchanging particles once per time step.

Every step of the method runs in the library's kernels (walk, packing by
tile, assembly of natives and ghosts, the mass transfer, dropping the
ghosts); this module only moves the packed records between processes with
``torch.distributed`` -- an all-to-all of the record counts, then one of the
records (NCCL on device buffers, or gloo through host copies) -- and keeps
the send buffer large enough.
"""
from __future__ import annotations

import numpy as np

from . import mtpt


def _order_key(x) -> np.ndarray:
    """int64 image of binary64 values that orders like the values (-0 below +0)."""
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.int64)
    return b ^ ((b >> 63) & np.int64(0x7FFFFFFFFFFFFFFF))


def tile_of(pos, lo, hi, tiles) -> np.ndarray:
    """Tile of each particle (pos: dim x n), numbered t0 + f0 (t1 + f1 t2):
    along axis a the edges are e_t = lo_a + t width_a (width_a = (hi_a - lo_a)
    / f_a) and a coordinate lies in tile t when e_t <= x < e_(t+1), the first
    and last tiles open-ended -- the library's rule, on the same binary64
    edges compared through the same order keys, for handing each process its
    natives."""
    pos = np.asarray(pos, dtype=np.float64)
    t = np.zeros(pos.shape[1], dtype=np.int64)
    mult = 1
    for a in range(pos.shape[0]):
        f = int(tiles[a])
        width = (hi[a] - lo[a]) / f
        edges = lo[a] + np.arange(f + 1, dtype=np.float64) * width
        t += np.searchsorted(_order_key(edges[1:f]), _order_key(pos[a]), side="right") * mult
        mult *= f
    return t


class Subdomain:
    """This process's tile of a run of n_global particles.

    params: the run's Params (the whole box); pos, mass, ids: this tile's
    natives (dim x n SoA, n, n global generator ids); dist: the initialised
    torch.distributed module, one process per tile (rank = tile).  ``lib``
    and ``device`` default to the CUDA library and device memory; the tests
    of the exchange alone pass a stand-in and "cpu"."""

    def __init__(self, params: mtpt.Params, n_global: int, pos, mass, ids, dist, tiles=None,
                 lib=mtpt, device: str = "cuda"):
        import torch
        self.lib = lib
        self.device = device
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        self.dim = params.dim
        self.k = params.dim + 2                      # values per record
        self.tiles = tuple(tiles) if tiles is not None else \
            lib.mtpt_tiling_factors(params.dim, params.lo, params.hi, self.world)
        if int(np.prod(self.tiles)) != self.world:
            raise ValueError(f"{self.tiles} tiles for {self.world} processes")
        self.nccl = dist.get_backend() == "nccl"
        self.h = lib.mtpt_create(params)
        if device == "cuda":
            lib.mtpt_set_stream(self.h, torch.cuda.current_stream().cuda_stream)
        lib.mtpt_set_tiling(self.h, self.tiles, self.rank, n_global)
        lib.mtpt_set_particles_tile(self.h, self.dim, pos, mass, ids)
        n = len(np.asarray(mass).ravel())
        self.send = torch.empty((max(1024, n // 4), self.k), dtype=torch.float64, device=device)

    def _all_to_all(self, send, send_split, recv_split):
        """Records of every tile for every other: NCCL moves device buffers,
        gloo host copies."""
        import torch
        comm = self.device if self.nccl else "cpu"
        recv = torch.empty((int(sum(recv_split)), self.k), dtype=torch.float64, device=comm)
        src = send if send.device.type == comm else send.to(comm)
        self.dist.all_to_all_single(recv, src, list(recv_split), list(send_split))
        return recv if recv.device.type == self.device else recv.to(self.device)

    def step(self, nsteps: int = 1) -> None:
        import torch
        lib = self.lib
        comm = self.device if self.nccl else "cpu"
        for _ in range(nsteps):
            lib.mtpt_step_ex(self.h, 1, mtpt.MTPT_DO_WALK)
            rc, counts = lib.mtpt_tile_pack(self.h, self.send, self.world)
            per = counts[0::2] + counts[1::2]
            per[self.rank] = 0                       # this tile's share stays with it
            if rc == mtpt.MTPT_ERR_CAPACITY:
                self.send = torch.empty((int(per.sum() * 5 // 4) + 1024, self.k),
                                        dtype=torch.float64, device=self.device)
                rc, counts = lib.mtpt_tile_pack(self.h, self.send, self.world)
                if rc != mtpt.MTPT_OK:
                    raise mtpt.MtptError(rc, "mtpt_tile_pack")
            send_split = torch.tensor(per, dtype=torch.int64, device=comm)
            recv_split = torch.empty_like(send_split)
            self.dist.all_to_all_single(recv_split, send_split)
            total = int(per.sum())
            recv = self._all_to_all(self.send[:total], per.tolist(), recv_split.tolist())
            lib.mtpt_tile_transfer(self.h, recv)

    def natives(self):
        """(ids, positions dim x n, masses) of this tile's natives."""
        lib = self.lib
        n = lib.mtpt_get_info(self.h)["n"]
        return (lib.mtpt_get_ids(self.h, n), lib.mtpt_get_positions(self.h, self.dim, n),
                lib.mtpt_get_masses(self.h, n))

    def info(self) -> dict:
        return self.lib.mtpt_get_info(self.h)

    def close(self) -> None:
        if self.h is not None:
            self.lib.mtpt_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
