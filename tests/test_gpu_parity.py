"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bars: positions of the random walk and neighbour pair sets bit-exact; masses
within 1e-12 (binary64 form) or 1e-5 (precision form) of max |M| of the
oracle; pair counts exact.  Sizes span many cells, several thread blocks and
ragged tails."""
import numpy as np
import pytest

import oracle as O
from paper_2204_03756_gb300 import mtpt, workloads

from gpu_helpers import TOL, oracle_params, params_of, rel_err, run_both

pytestmark = pytest.mark.gpu

FORMS = [mtpt.MTPT_FP64, mtpt.MTPT_FP32W]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available()
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()


def test_walk_is_bit_exact_with_the_oracle():
    w = workloads.get("heaviside_2d", 10_001)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, kappa=1.0, D=2.0)          # pure walk, no transfer
    g, r = run_both(p, pos, mass, 7)
    assert np.array_equal(g["pos"], r["pos"])
    assert np.array_equal(g["mass"], mass)
    assert g["info"]["pair_count"] == 0 and g["info"]["step"] == 7


@pytest.mark.parametrize("seed,step", [(0, 0), (2 ** 64 - 1, 2 ** 64 - 1), (2204037561, 2 ** 32 + 9)])
def test_walk_takes_its_normals_from_the_library_generator(seed, step):
    """Hand-picked ids, seeds and steps (counter (id, step lo, step hi, 0),
    key = seed): each GPU move equals sigma z with z the Box-Muller normals of
    the words that a third-party Philox4x32-10 gives for that counter."""
    from philox_library import philox4x32_10 as library_philox
    ids = np.array([0, 1, 2, 3, 31, 32, 255, 256, 1000], dtype=np.uint32)
    n = ids.size
    p = mtpt.Params(dim=3, D=2.0, kappa=1.0, dt=0.1, lo=(0.0,) * 3, hi=(100.0,) * 3, seed=seed)
    total = int(ids.max()) + 1                 # particle i carries generator id i
    with mtpt.Simulation(p, np.full((3, total), 50.0), np.ones(total)) as sim:
        sim.set_step(step)
        sim.step(1)
        got = sim.positions()[:, ids]
    ctr = np.stack([ids, np.full(n, step & 0xFFFFFFFF, np.uint32),
                    np.full(n, step >> 32, np.uint32), np.zeros(n, np.uint32)], axis=1)
    z = O.box_muller(library_philox(ctr, [seed & 0xFFFFFFFF, seed >> 32]))
    sigma = np.sqrt(2.0 * 2.0 * 0.1)
    want = 50.0 + sigma * z[:, :3].T.astype(np.float64)   # one rounding each, no fma
    assert np.all(np.abs(want - 50.0) < 50.0)              # no wall reached
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_walk_with_walls_bit_exact_3d(dim):
    rng = np.random.default_rng(dim)
    n = 3000
    lo, hi = (0.0,) * dim, (3.0,) * dim          # small box: many reflections
    pos = rng.uniform(0, 3.0, size=(dim, n))
    pos[:, :10] = 0.0
    pos[:, 10:20] = 3.0
    p = mtpt.Params(dim=dim, D=1.0, kappa=0.5, dt=0.2, lo=lo, hi=hi, seed=17)
    g, r = run_both(p, pos, np.zeros(n), 5)
    assert np.array_equal(g["pos"], r["pos"])


def _pairs_gpu(p, pos):
    with mtpt.Simulation(p, pos, np.zeros(pos.shape[1])) as sim:
        return sim.pairs()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("dim,n,L", [(1, 1999, 400.0), (2, 2000, 30.0), (3, 1777, 9.0)])
def test_pair_sets_bit_exact_vs_brute_force(form, dim, n, L):
    rng = np.random.default_rng(100 + dim)
    pos = rng.uniform(0, L, size=(dim, n))
    pos[:, :40] = np.round(pos[:, :40])          # lattice points and duplicates
    pos[0, 40:60] = 0.0                          # on the wall
    pos[:, 60:70] = pos[:, 70:80]                # coincident pairs
    p = mtpt.Params(dim=dim, D=1.0, kappa=0.5, dt=0.1, lo=(0.0,) * dim, hi=(L,) * dim,
                    seed=1, precision=form)
    gi, gj = _pairs_gpu(p, pos)
    psi2 = O.derived(oracle_params(p))["psi2"]
    bi, bj = O.pairs(pos, psi2, "brute")
    assert np.array_equal(gi, bi) and np.array_equal(gj, bj)


def _pairs_gpu_tuned(p, pos, cell_scale):
    with mtpt.Simulation(p, pos, np.zeros(pos.shape[1])) as sim:
        sim.set_tuning(cell_scale, 256)
        return sim.pairs()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("dim,n,L", [(1, 1999, 400.0), (2, 2000, 30.0), (3, 1777, 9.0)])
def test_pair_sets_with_half_width_cells_bit_exact_vs_brute_force(form, dim, n, L):
    """Cells half the cutoff wide (neighbours up to two cells away per axis)
    find the same pairs as brute force, lattice points, walls and coincident
    particles included."""
    rng = np.random.default_rng(200 + dim)
    pos = rng.uniform(0, L, size=(dim, n))
    pos[:, :40] = np.round(pos[:, :40])
    pos[0, 40:60] = 0.0
    pos[:, 60:70] = pos[:, 70:80]
    p = mtpt.Params(dim=dim, D=1.0, kappa=0.5, dt=0.1, lo=(0.0,) * dim, hi=(L,) * dim,
                    seed=1, precision=form)
    gi, gj = _pairs_gpu_tuned(p, pos, 0.5)
    bi, bj = O.pairs(pos, O.derived(oracle_params(p))["psi2"], "brute")
    assert np.array_equal(gi, bi) and np.array_equal(gj, bj)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("name,n,steps", [("heaviside_2d", 20_003, 6), ("heaviside_3d", 30_001, 4)])
def test_half_width_cells_step_parity(form, name, n, steps):
    w = workloads.get(name, n)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=form)
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.set_tuning(0.5, 128)
        sim.step(steps)
        x, m, info = sim.positions(), sim.masses(), sim.info()
    xr, mr, npairs = O.run(oracle_params(p), pos, mass, steps)
    assert np.array_equal(x, xr)
    assert info["pair_count"] == npairs
    assert rel_err(m, mr) <= TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_pair_sets_on_exact_ties(form):
    # D_MT dt = 0.25 makes psi = lambda exactly; lambda = 1.25, psi^2 = 1.5625 and
    # 0.75^2 + 1^2 = 1.5625: these pairs sit exactly on the cutoff.
    p = mtpt.Params(dim=2, D=2.5, kappa=0.0, dt=0.1, lam=1.25, lo=(0, 0), hi=(20, 20),
                    seed=3, precision=form)
    d = O.derived(oracle_params(p))
    assert d["psi2"] == 1.5625
    base = np.array([[2.0, 2.75, 10.0, 10.75, 10.0 + 1.25, 15.0, 15.0],
                     [2.0, 3.0, 10.0, 11.0, 10.0, 15.0, np.nextafter(16.25, 20.0)]])
    bi, bj = O.pairs(base, d["psi2"], "brute")
    for gi, gj in (_pairs_gpu(p, base), _pairs_gpu_tuned(p, base, 0.5)):
        assert np.array_equal(gi, bi) and np.array_equal(gj, bj)
        got = set(zip(gi.tolist(), gj.tolist()))
        assert (0, 1) in got and (2, 3) in got and (2, 4) in got and (5, 6) not in got


@pytest.mark.parametrize("form", FORMS)
def test_pair_sets_large_vs_kdtree(form):
    w = workloads.get("heaviside_3d", 60_000)
    pos, _ = workloads.initial_state(w)
    p = params_of(w, precision=form)
    gi, gj = _pairs_gpu(p, pos)
    ki, kj = O.pairs(pos, O.derived(oracle_params(p))["psi2"], "kdtree")
    assert np.array_equal(gi, ki) and np.array_equal(gj, kj)


@pytest.mark.parametrize("form", FORMS)
def test_row_sums_match_the_oracle(form):
    w = workloads.get("heaviside_2d", 5003)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=form, kappa=0.0)  # transfer only: positions fixed
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.step(1)
        rs = sim.row_sums()
        m = sim.masses()
    m_ref, rs_ref, cs_ref, _ = O.mass_transfer(oracle_params(p), pos, mass)
    tol = 1e-13 if form == mtpt.MTPT_FP64 else 3e-6
    assert rel_err(rs, rs_ref) <= tol
    assert rel_err(m, m_ref) <= TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_heaviside_2d_full_config_masses(form):
    """The 2-d plain-diffusion workload in full: N = 10,000, 100 steps."""
    w = workloads.get("heaviside_2d")
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=form)
    g, r = run_both(p, pos, mass, w.steps)
    assert np.array_equal(g["pos"], r["pos"])
    assert g["info"]["pair_count"] == r["pairs"]
    err = rel_err(g["mass"], r["mass"])
    assert err <= TOL[form], err
    drift = abs(g["mass"].sum() - mass.sum()) / mass.sum()
    assert drift < 1e-12, drift


@pytest.mark.parametrize("form", FORMS)
def test_heaviside_3d_scaled_masses(form):
    w = workloads.get("heaviside_3d", 20_000)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=form)
    g, r = run_both(p, pos, mass, 20)
    assert np.array_equal(g["pos"], r["pos"])
    assert g["info"]["pair_count"] == r["pairs"]
    assert rel_err(g["mass"], r["mass"]) <= TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_gaussian_and_uniform_mass_workloads_scaled(form):
    for name, n, steps in (("gaussian_2d", 40_000, 10), ("uniform_mass_2d", 30_000, 10)):
        w = workloads.get(name, n)
        pos, mass = workloads.initial_state(w)
        p = params_of(w, precision=form)
        g, r = run_both(p, pos, mass, steps)
        assert np.array_equal(g["pos"], r["pos"])
        assert rel_err(g["mass"], r["mass"]) <= TOL[form], name


def test_one_dimensional_run():
    rng = np.random.default_rng(9)
    n = 4097
    pos = rng.uniform(0, 500.0, size=(1, n))
    mass = (pos[0] < 250).astype(float)
    for form in FORMS:
        p = mtpt.Params(dim=1, D=1.0, kappa=0.5, dt=0.1, lo=(0.0,), hi=(500.0,), seed=5,
                        precision=form)
        g, r = run_both(p, pos, mass, 30)
        assert np.array_equal(g["pos"], r["pos"])
        assert rel_err(g["mass"], r["mass"]) <= TOL[form]


def test_uniform_masses_stay_uniform_bit_exactly():
    w = workloads.get("heaviside_2d", 7000)
    pos, _ = workloads.initial_state(w)
    mass = np.full(w.n, 0.375)
    for form in FORMS:
        with mtpt.Simulation(params_of(w, precision=form), pos, mass) as sim:
            sim.step(5)
            assert np.array_equal(sim.masses(), mass)


def test_transfer_only_keeps_positions_and_walk_only_keeps_masses():
    w = workloads.get("heaviside_2d", 3000)
    pos, mass = workloads.initial_state(w)
    with mtpt.Simulation(params_of(w), pos, mass) as sim:
        sim.step(3, flags=mtpt.MTPT_DO_TRANSFER)
        assert np.array_equal(sim.positions(), pos)
        assert sim.info()["step"] == 0
        m3 = sim.masses()
        sim.step(2, flags=mtpt.MTPT_DO_WALK)
        assert np.array_equal(sim.masses(), m3)
        assert sim.info()["step"] == 2


def test_runs_are_bit_reproducible():
    w = workloads.get("gaussian_2d", 50_000)
    pos, mass = workloads.initial_state(w)
    outs = []
    for _ in range(2):
        with mtpt.Simulation(params_of(w), pos, mass) as sim:
            sim.step(6)
            outs.append((sim.masses(), sim.positions()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_checkpoint_resume_is_bit_identical():
    w = workloads.get("heaviside_2d", 6000)
    pos, mass = workloads.initial_state(w)
    p = params_of(w)
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.step(10)
        full_m, full_x = sim.masses(), sim.positions()
    with mtpt.Simulation(p, pos, mass) as sim:
        sim.step(4)
        mid_m, mid_x = sim.masses(), sim.positions()
    with mtpt.Simulation(p, mid_x, mid_m) as sim:
        sim.set_step(4)
        sim.step(6)
        assert np.array_equal(sim.masses(), full_m)
        assert np.array_equal(sim.positions(), full_x)


def test_edge_cases_empty_single_and_one_cell():
    p = mtpt.Params(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0, 0), hi=(10, 10), seed=2)
    with mtpt.Simulation(p, np.zeros((2, 0)), np.zeros(0)) as sim:
        sim.step(3)
        assert sim.masses().size == 0
        assert sim.info()["pair_count"] == 0
    with mtpt.Simulation(p, np.array([[5.0], [5.0]]), np.array([2.0])) as sim:
        sim.step(3)
        assert np.array_equal(sim.masses(), [2.0])
    # every particle in one cell (box smaller than the cutoff): all pairs
    rng = np.random.default_rng(4)
    n = 700
    q = mtpt.Params(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0, 0), hi=(0.9, 0.9), seed=2)
    pos = rng.uniform(0, 0.9, size=(2, n))
    mass = rng.uniform(0, 1, n)
    with mtpt.Simulation(q, pos, mass) as sim:
        assert sim.info()["cells"][:2] == (1, 1)
    for form in FORMS:       # every particle has n - 1 neighbours: list overflow path
        qf = mtpt.Params(**{**q.__dict__, "precision": form})
        g, r = run_both(qf, pos, mass, 3, method="brute")
        assert np.array_equal(g["pos"], r["pos"])
        assert g["info"]["pair_count"] == r["pairs"] == 3 * n * (n - 1)
        assert rel_err(g["mass"], r["mass"]) <= TOL[form]


def test_neighbour_lists_with_mixed_overflow_match_the_oracle():
    # a dense clump (many neighbours: over the list capacity) inside a sparse
    # box (few neighbours): both pass-2 paths in one launch
    rng = np.random.default_rng(12)
    sparse = rng.uniform(0, 60.0, size=(2, 3000))
    clump = 30.0 + rng.uniform(-0.4, 0.4, size=(2, 150))
    pos = np.concatenate([sparse, clump], axis=1)
    mass = rng.uniform(0, 1, pos.shape[1])
    p = mtpt.Params(dim=2, D=1.0, kappa=0.5, dt=0.1, lo=(0, 0), hi=(60, 60), seed=8,
                    precision=mtpt.MTPT_FP32W)
    g, r = run_both(p, pos, mass, 4)
    assert np.array_equal(g["pos"], r["pos"])
    assert g["info"]["pair_count"] == r["pairs"]
    assert rel_err(g["mass"], r["mass"]) <= TOL[mtpt.MTPT_FP32W]


def test_ragged_sizes_around_block_boundaries():
    for n in (1, 2, 255, 256, 257, 511, 513):
        ww = workloads.get("heaviside_2d", n)
        pos, mass = workloads.initial_state(ww)
        p = params_of(ww)
        g, r = run_both(p, pos, mass, 4, method="brute")
        assert np.array_equal(g["pos"], r["pos"])
        assert rel_err(g["mass"], r["mass"]) <= 1e-12


def test_device_buffers_through_torch():
    import torch
    w = workloads.get("heaviside_2d", 9000)
    pos, mass = workloads.initial_state(w)
    p = params_of(w)
    h = mtpt.mtpt_create(p)
    try:
        pt = torch.from_numpy(pos.copy()).cuda()
        mt = torch.from_numpy(mass.copy()).cuda()
        mtpt.mtpt_set_particles_device(h, 2, pt, mt)
        mtpt.mtpt_step(h, 5)
        out_m = torch.empty(w.n, dtype=torch.float64, device="cuda")
        out_x = torch.empty(2 * w.n, dtype=torch.float64, device="cuda")
        mtpt.mtpt_get_masses_device(h, out_m)
        mtpt.mtpt_get_positions_device(h, out_x)
        mtpt.mtpt_sync(h)
        torch.cuda.synchronize()
        xr, mr, _ = O.run(oracle_params(p), pos, mass, 5)
        assert np.array_equal(out_x.cpu().numpy().reshape(2, -1), xr)
        assert rel_err(out_m.cpu().numpy(), mr) <= 1e-12
        # a device-side domain violation is latched and reported at the next sync
        bad = pt.clone()
        bad[0, 0] = 1e9
        mtpt.mtpt_set_particles_device(h, 2, bad, mt)
        with pytest.raises(mtpt.MtptError) as e:
            mtpt.mtpt_sync(h)
        assert e.value.code == mtpt.MTPT_ERR_OUT_OF_DOMAIN
    finally:
        mtpt.mtpt_destroy(h)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("case", ["far_f32_cells", "farther_f32_cells", "far_f64_cells",
                                  "sparse_wide_cells", "one_cell_high", "on_cell_corners"])
def test_pair_windows_on_adversarial_boxes(form, case):
    """The per-row candidate windows rest on a slack derived from the
    binary32 cell-index and offset error bounds: boxes far from the origin
    (binary32 cell indices near their limit, and binary64 ones beyond it),
    cells much wider than psi, a single cell row and particles on cell
    corners must all keep the exact pair set -- in the emitted pairs and in
    the pair counts of both pair passes."""
    cases = ["far_f32_cells", "far_f64_cells", "sparse_wide_cells", "one_cell_high",
             "on_cell_corners", "farther_f32_cells"]
    rng = np.random.default_rng(11 + cases.index(case))
    n = 2500
    if case == "far_f32_cells":
        lo = np.array([4800.0, -5000.0]); L = np.array([45.0, 38.0])
    elif case == "farther_f32_cells":             # binary32 cell error ~5e-3 cells
        lo = np.array([48000.0, -50000.0]); L = np.array([45.0, 38.0])
    elif case == "far_f64_cells":
        lo = np.array([2.0e6, -3.5e6]); L = np.array([45.0, 38.0])
    elif case == "sparse_wide_cells":              # cells ~14 psi wide (count capped)
        n = 40
        lo = np.array([0.0, 0.0]); L = np.array([200.0, 150.0])
    elif case == "one_cell_high":
        lo = np.array([0.0, 0.0]); L = np.array([900.0, 1.0])
    else:
        lo = np.array([0.0, 0.0]); L = np.array([30.0, 30.0])
    pos = lo[:, None] + rng.uniform(0, 1, size=(2, n)) * L[:, None]
    p = mtpt.Params(dim=2, D=1.0, kappa=0.0, dt=0.1, lo=tuple(lo), hi=tuple(lo + L),
                    seed=9, precision=form)
    if case == "sparse_wide_cells":
        pos[:, :20] = lo[:, None] + np.array([[30.0], [40.0]]) + rng.uniform(0, 3, size=(2, 20))
    if case == "on_cell_corners":
        psi = O.derived(oracle_params(p))["psi"]
        ncell = np.floor(L / (psi * (1 + 1e-6)))
        w = L / ncell
        k = rng.integers(0, ncell[0], size=400), rng.integers(0, ncell[1], size=400)
        pos[0, :400] = lo[0] + k[0] * w[0]
        pos[1, :400] = lo[1] + k[1] * w[1]
        pos[:, 400:800] = pos[:, :400] + rng.choice([-1e-12, 0.0, 1e-12], size=(2, 400))
        pos = np.clip(pos, lo[:, None], (lo + L)[:, None])
    psi2 = O.derived(oracle_params(p))["psi2"]
    bi, bj = O.pairs(pos, psi2, "brute")
    gi, gj = _pairs_gpu(p, pos)
    assert np.array_equal(gi, bi) and np.array_equal(gj, bj)
    with mtpt.Simulation(p, pos, rng.uniform(0, 1, n)) as sim:
        sim.step(1)                                    # kappa = 0: transfer only
        assert sim.info()["pair_count"] == len(bi)


# --- advection (the velocity term of the model equation, Sec. 2) ------------------

@pytest.mark.parametrize("dim", [1, 2, 3])
def test_advected_walk_is_bit_exact_with_reflections(dim):
    """v dt + sigma xi per axis before the reflection, as in the oracle; a
    small box and a large velocity force repeated mirrors at the walls, and an
    axis with v = 0 keeps the plain walk."""
    rng = np.random.default_rng(40 + dim)
    n = 3001
    L = 6.0
    pos = rng.uniform(0, L, size=(dim, n))
    v = (2.5, 0.0, -4.0)[:dim]
    for form in FORMS:
        p = mtpt.Params(dim=dim, D=1.0, kappa=0.5, dt=0.2, lo=(0.0,) * dim, hi=(L,) * dim,
                        seed=23, precision=form, v=v)
        g, r = run_both(p, pos, rng.uniform(0, 1, n), 6)
        assert np.array_equal(g["pos"], r["pos"])
        assert g["info"]["pair_count"] == r["pairs"]
        assert rel_err(g["mass"], r["mass"]) <= TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_advection_workload_scaled_matches_the_oracle(form):
    w = workloads.get("advection_2d", 40_000)
    pos, mass = workloads.initial_state(w)
    g, r = run_both(params_of(w, precision=form), pos, mass, 10)
    assert np.array_equal(g["pos"], r["pos"])
    assert g["info"]["pair_count"] == r["pairs"]
    assert rel_err(g["mass"], r["mass"]) <= TOL[form]


def test_walk_without_random_walk_still_advects():
    """kappa = 0 switches the random walk off but not the advection."""
    rng = np.random.default_rng(44)
    pos = rng.uniform(100, 200, size=(2, 2000))
    p = mtpt.Params(dim=2, D=1.0, kappa=0.0, dt=0.1, lo=(0, 0), hi=(300, 300), seed=3,
                    v=(1.5, -0.5))
    g, r = run_both(p, pos, rng.uniform(0, 1, 2000), 4)
    assert np.array_equal(g["pos"], r["pos"])
    assert not np.array_equal(g["pos"], pos)
