"""Host side of the split domain (Secs. 4-5), without a GPU: the checkerboard
factors of Eq. "minimization" from the C library, and the per-step exchange
of ddc.Subdomain run by gloo ranks on CPU around a stand-in tile."""
import os
import socket

import numpy as np
import pytest

from paper_2204_03756_gb300 import build as cuda_build
from paper_2204_03756_gb300 import ddc, mtpt


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return mtpt.load()


def _pairs_by_eq_minimization(n, A):
    """Every (f1, f2), f1 <= f2, f1 f2 = n, with |f2 / f1 - A| least."""
    cand = [(f1, n // f1) for f1 in range(1, n + 1) if n % f1 == 0 and f1 <= n // f1]
    best = min(abs(f2 / f1 - A) for f1, f2 in cand)
    return [(f1, f2) for f1, f2 in cand if abs(f2 / f1 - A) == best]


@pytest.mark.parametrize("W,H", [(100.0, 100.0), (150.0, 100.0), (370.0, 100.0),
                                 (100.0, 250.0), (1000.0, 1000.0)])
def test_tiling_factors_follow_eq_minimization(lib, W, H):
    for n in range(1, 97):
        f = mtpt.mtpt_tiling_factors(2, (0.0, 0.0), (W, H), n)
        assert f[2] == 1 and f[0] * f[1] == n
        A = max(W, H) / min(W, H)
        wide, short = (f[0], f[1]) if W >= H else (f[1], f[0])
        assert (short, wide) in _pairs_by_eq_minimization(n, A), (n, f)
        # among equally good pairs, the smallest f1
        assert short == min(p[0] for p in _pairs_by_eq_minimization(n, A))
    # a prime number of tiles reverts to slices along the longer side (Sec. 4.2)
    f = mtpt.mtpt_tiling_factors(2, (0.0, 0.0), (W, H), 7)
    assert sorted(f[:2]) == [1, 7] and (f[0] == 7) == (W >= H)


def test_tiling_factors_3d_and_1d(lib):
    for n in (1, 2, 4, 6, 8, 12, 27, 30, 64):
        for L in ((100.0, 100.0, 100.0), (200.0, 100.0, 50.0)):
            f = mtpt.mtpt_tiling_factors(3, (0.0,) * 3, L, n)
            assert f[0] * f[1] * f[2] == n
            ratio = lambda g: max(L[a] / g[a] for a in range(3)) / min(L[a] / g[a] for a in range(3))
            best = min(ratio((a, b, n // (a * b))) for a in range(1, n + 1) for b in range(1, n + 1)
                       if n % a == 0 and (n // a) % b == 0)
            assert ratio(f) == best
    assert mtpt.mtpt_tiling_factors(1, (0.0,), (10.0,), 5) == (5, 1, 1)
    assert mtpt.mtpt_tiling_factors(3, (0.0,) * 3, (126.0,) * 3, 8) == (2, 2, 2)


def test_tile_of_matches_the_ownership_rule():
    lo, hi, tiles = (0.0, -5.0), (100.0, 5.0), (4, 2)
    pos = np.array([[0.0, 24.999, 25.0, 99.0, 100.0, 50.0],
                    [-5.0, 0.0, -0.001, 5.0, 4.0, 0.0]])
    assert ddc.tile_of(pos, lo, hi, tiles).tolist() == [0, 4, 1, 7, 7, 6]
    # an edge at zero: -0 sorts below it (the order keys), +0 on it
    z = np.array([[-0.0, 0.0, -1e-300, 1e-300]])
    assert ddc.tile_of(z, (-100.0,), (100.0,), (2,)).tolist() == [0, 1, 0, 1]


# --- the exchange, gloo ranks on CPU around a stand-in tile -------------------

BOX = 100.0
SHIFT = 7.0          # every walk moves each particle this far in x (wrapping)
PAD = 3.0            # a stand-in ghost: copy for the right tile within PAD of its edge


class _StandInTile:
    """Records of dim + 2 values on the host: slab tiles along x, a fixed
    shift as the walk, and ghost copies for the tile to the right; enough to
    drive Subdomain's counts, splits, buffer growth and all-to-all."""

    def __init__(self):
        self.ghosts_seen = 0

    def mtpt_tiling_factors(self, dim, lo, hi, ntiles):
        return (ntiles, 1, 1)

    def mtpt_create(self, params):
        return {"dim": params.dim}

    def mtpt_set_tiling(self, h, tiles, tile, n_global):
        h.update(P=int(np.prod(tiles)), rank=tile, width=BOX / tiles[0])

    def mtpt_set_particles_tile(self, h, dim, pos, mass, ids):
        h["rec"] = np.column_stack([np.asarray(pos).T, mass, np.asarray(ids, np.float64)])

    def mtpt_step_ex(self, h, nsteps, flags):
        assert flags == mtpt.MTPT_DO_WALK
        h["rec"][:, 0] = (h["rec"][:, 0] + SHIFT) % BOX

    def _owner(self, h, x):
        return np.minimum((x // h["width"]).astype(int), h["P"] - 1)

    def mtpt_tile_pack(self, h, send, P):
        rec = h["rec"]
        own = self._owner(h, rec[:, 0])
        right = own + 1
        ghost = (right < P) & ((own + 1) * h["width"] - rec[:, 0] < PAD)
        counts = np.zeros(2 * P, np.int64)
        parts = []
        for t in range(P):
            nat, gh = rec[own == t], rec[ghost & (right == t)]
            counts[2 * t], counts[2 * t + 1] = len(nat), len(gh)
            if t == h["rank"]:
                h["keep"] = nat
            else:
                parts += [nat, gh]
        out = np.concatenate(parts) if parts else np.zeros((0, rec.shape[1]))
        if len(out) > send.shape[0]:
            return mtpt.MTPT_ERR_CAPACITY, counts
        import torch
        send[:len(out)] = torch.from_numpy(out)
        return mtpt.MTPT_OK, counts

    def mtpt_tile_transfer(self, h, recv):
        r = recv.numpy()
        native = self._owner(h, r[:, 0]) == h["rank"]
        self.ghosts_seen += int((~native).sum())
        h["rec"] = np.concatenate([h["keep"], r[native]])

    def mtpt_get_info(self, h):
        return {"n": len(h["rec"]), "pair_count": 0}

    def mtpt_get_ids(self, h, n):
        return h["rec"][:, -1].astype(np.uint32)

    def mtpt_get_positions(self, h, dim, n):
        return h["rec"][:, :dim].T.copy()

    def mtpt_get_masses(self, h, n):
        return h["rec"][:, dim_of(h)].copy()

    def mtpt_destroy(self, h):
        pass


def dim_of(h):
    return h["dim"]


def _exchange_rank(rank, world, port, n_per, steps, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        rng = np.random.default_rng(5)
        n = n_per * world
        pos = np.vstack([rng.uniform(0, BOX, n), rng.uniform(0, 10.0, n)])
        ids = np.arange(n)
        stand_in = _StandInTile()
        mine = np.minimum((pos[0] // (BOX / world)).astype(int), world - 1) == rank
        p = mtpt.Params(dim=2, lo=(0.0, 0.0), hi=(BOX, 10.0))
        sd = ddc.Subdomain(p, n, pos[:, mine], ids[mine] * 0.5, ids[mine], dist,
                           lib=stand_in, device="cpu")
        sd.step(steps)
        got = sd.natives()
        everyone = [None] * world
        dist.all_gather_object(everyone, (got, stand_in.ghosts_seen, sd.send.shape[0]))
        if rank == 0:
            np.save(out, np.array(everyone, dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 4])
def test_exchange_moves_every_particle_to_its_tile(tmp_path, world):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    n_per, steps = 20_000, 5
    out = str(tmp_path / "tiles.npy")
    port = _free_port()
    procs = [ctx.Process(target=_exchange_rank, args=(r, world, port, n_per, steps, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    everyone = np.load(out, allow_pickle=True)
    rng = np.random.default_rng(5)
    n = n_per * world
    x0 = rng.uniform(0, BOX, n)
    seen = np.zeros(n, np.int64)
    for rank, ((ids, x, m), ghosts, cap) in enumerate(everyone):
        ids = ids.astype(np.int64)
        seen[ids] += 1
        want = x0[ids]
        for _ in range(steps):
            want = (want + SHIFT) % BOX
        assert np.array_equal(x[0], want)
        assert np.array_equal(m, ids * 0.5)
        owner = np.minimum((x[0] // (BOX / world)).astype(int), world - 1)
        assert np.all(owner == rank)
        assert ghosts > 0 or rank == 0             # the first tile has no left neighbour
    assert np.all(seen == 1)                       # every particle on exactly one tile
    if world == 4:                                 # a slab of 25 loses 28 % per step
        assert max(e[2] for e in everyone) > n_per // 4   # the send buffer grew
