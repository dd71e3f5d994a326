"""The split domain on the GPU (Secs. 4-5): P processes, one tile each, each
driving the library on this machine's GPU and exchanging particles through
gloo; after T steps the union of their natives is the single-domain run --
the same positions, masses and ordered pair count bit for bit (the tile's
cell grid is the undivided grid's part, its ghosts reach 2 psi) -- and
matches the oracle within the form's tolerance.  No kernel of one process
waits for another's: the exchange is host-side, between launches."""
import os
import socket
import zlib

import numpy as np
import pytest

import oracle as O
from paper_2204_03756_gb300 import ddc, mtpt

from gpu_helpers import TOL, oracle_params, rel_err

pytestmark = pytest.mark.gpu

# name: (dim, n, box side, D, kappa, dt, tiles, steps, form, mass kind)
CASES = {
    "2d_2x2_fp64": (2, 40_000, 200.0, 1.0, 0.5, 0.1, 4, 8, mtpt.MTPT_FP64, "heaviside"),
    "2d_2x2_fp32w": (2, 40_000, 200.0, 1.0, 0.5, 0.1, 4, 8, mtpt.MTPT_FP32W, "heaviside"),
    "2d_3x2_dense": (2, 5_400, 30.0, 2.0, 0.5, 0.1, 6, 12, mtpt.MTPT_FP64, "uniform"),
    "3d_2x2x1_fp32w": (3, 30_000, 31.0, 1.0, 0.5, 0.05, 4, 6, mtpt.MTPT_FP32W, "heaviside"),
    "3d_2x1x1_fp64": (3, 20_000, 27.0, 1.0, 0.5, 0.05, 2, 6, mtpt.MTPT_FP64, "uniform"),
    "1d_3_fp64": (1, 3_000, 3_000.0, 1.0, 0.5, 0.1, 3, 10, mtpt.MTPT_FP64, "heaviside"),
}


def _setup(name):
    dim, n, L, D, kappa, dt, world, steps, form, kind = CASES[name]
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    pos = rng.uniform(0.0, L, size=(dim, n))
    pos[:, :4] = L / 2                       # particles on tile edges (L / 2 is one for P = 2, 4)
    pos[0, 4:8] = (0.0, L, L / 3, 2 * L / 3)
    mass = (pos[0] < L / 2).astype(np.float64) if kind == "heaviside" else rng.uniform(0, 1, n)
    p = mtpt.Params(dim=dim, D=D, kappa=kappa, dt=dt, lo=(0.0,) * dim, hi=(L,) * dim,
                    seed=2204 + dim, precision=form)
    return p, pos, mass, world, steps


def _tile_rank(rank, world, port, name, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2204_03756_gb300 import build
        build.build()
        p, pos, mass, world, steps = _setup(name)
        tiles = mtpt.mtpt_tiling_factors(p.dim, p.lo, p.hi, world)
        mine = ddc.tile_of(pos, p.lo, p.hi, tiles) == rank
        ids = np.flatnonzero(mine).astype(np.uint32)
        with ddc.Subdomain(p, pos.shape[1], pos[:, mine], mass[mine], ids, dist) as sd:
            sd.step(steps)
            got_ids, x, m = sd.natives()
            pairs = sd.info()["pair_count"]
        np.savez(os.path.join(out_dir, f"tile{rank}.npz"), ids=got_ids, x=x, m=m, pairs=pairs,
                 tiles=np.array(tiles))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run_tiles(name, tmp_path):
    import multiprocessing as mp
    world = CASES[name][6]
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_tile_rank, args=(r, world, port, name, str(tmp_path)))
             for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=300)
    for pr in procs:
        if pr.is_alive():
            pr.kill()
    assert all(pr.exitcode == 0 for pr in procs), [pr.exitcode for pr in procs]
    return [np.load(os.path.join(tmp_path, f"tile{r}.npz")) for r in range(world)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()


@pytest.mark.parametrize("name", list(CASES))
def test_split_domain_equals_the_single_domain(name, tmp_path):
    p, pos, mass, world, steps = _setup(name)
    n = pos.shape[1]
    tiles = _run_tiles(name, tmp_path)
    x = np.full((p.dim, n), np.nan)
    m = np.full(n, np.nan)
    seen = np.zeros(n, np.int64)
    pairs = 0
    for r, t in enumerate(tiles):
        ids = t["ids"].astype(np.int64)
        assert np.all(ddc.tile_of(t["x"], p.lo, p.hi, tuple(t["tiles"])) == r)   # natives only
        seen[ids] += 1
        x[:, ids] = t["x"]
        m[ids] = t["m"]
        pairs += int(t["pairs"])
    assert np.all(seen == 1)                 # every particle native to exactly one tile
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.step(steps)
        xs, ms, info = sim.positions(), sim.masses(), sim.info()
    assert np.array_equal(x, xs)
    assert pairs == info["pair_count"]
    assert np.array_equal(m, ms)             # the same sums in the same order
    xr, mr, npairs = O.run(oracle_params(p), pos, mass, steps)
    assert np.array_equal(x, xr)
    assert pairs == npairs
    assert rel_err(m, mr) <= TOL[p.precision]
    # the run moved particles between tiles and filled pads
    moved = ddc.tile_of(x, p.lo, p.hi, tuple(tiles[0]["tiles"])) != \
        ddc.tile_of(pos, p.lo, p.hi, tuple(tiles[0]["tiles"]))
    assert moved.any()
