"""The hand-written adjoint (gradients of a binned-concentration misfit with
respect to the initial masses and D): dL/dM_0 against the oracle's reverse
sweep (the paper's transfer operator is symmetric, so applying the oracle's
own update to the adjoint vector is its transpose), dL/dD against central
finite differences of the oracle run in binary64 (same random path), and the
torch.autograd.Function end to end."""
import numpy as np
import pytest

import oracle as O
from paper_2204_03756_gb300 import mtpt, workloads

from gpu_helpers import oracle_params, params_of, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2204_03756_gb300 import build
    build.build()
    mtpt.load()


NB = (8, 8)


def _case(n=2000, steps=20, precision=mtpt.MTPT_FP64, v=(0.0, 0.0)):
    w = workloads.get("uniform_mass_2d", n)
    pos, mass = workloads.initial_state(w)
    p = params_of(w, precision=precision, v=v)
    target = workloads.target_field(NB, w.lo, w.hi)
    return w, p, pos, mass, target, steps


def _bins(w, x):
    ix = np.clip(((x[0] - w.lo[0]) / (w.hi[0] - w.lo[0]) * NB[0]).astype(int), 0, NB[0] - 1)
    iy = np.clip(((x[1] - w.lo[1]) / (w.hi[1] - w.lo[1]) * NB[1]).astype(int), 0, NB[1] - 1)
    return ix * NB[1] + iy


def _loss_and_grad(w, x, m, target):
    area = (w.hi[0] - w.lo[0]) / NB[0] * (w.hi[1] - w.lo[1]) / NB[1]
    b = _bins(w, x)
    C = np.bincount(b, weights=m, minlength=NB[0] * NB[1]) / area
    diff = C - target.ravel()
    return float((diff ** 2).sum()), 2.0 * diff[b] / area, b


def _oracle_forward(op, pos, mass, steps):
    ids = np.arange(mass.size, dtype=np.uint32)
    xs, x, m, pairs = [], pos, mass, 0
    for t in range(steps):
        x = O.random_walk(op, x, ids, t)
        m, _, _, np_ = O.mass_transfer(op, x, m)
        xs.append(x)
        pairs += np_
    return xs, x, m, pairs


@pytest.mark.parametrize("v", [(0.0, 0.0), (0.8, -0.3)])
def test_mass_gradient_matches_the_oracle_reverse_sweep_and_D_gradient_matches_fd(v):
    """Also with a velocity: advection moves the path (and so the operator
    A_t) but not the tangents dX/dD."""
    import torch
    w, p, pos, mass, target, steps = _case(v=v)
    op = oracle_params(p)
    xs, xT, mT, _ = _oracle_forward(op, pos, mass, steps)
    L, g, _ = _loss_and_grad(w, xT, mT, target)
    lam = g.copy()
    for t in reversed(range(steps)):
        lam = O.mass_transfer(op, xs[t], lam)[0]
    # GPU adjoint through the C ABI
    h = mtpt.mtpt_create(p)
    try:
        mtpt.mtpt_set_particles(h, 2, pos, mass)
        mtpt.mtpt_adjoint_forward(h, steps, 6)           # segments of 6, 6, 6, 2
        xg, mg = mtpt.mtpt_get_positions(h, 2, w.n), mtpt.mtpt_get_masses(h, w.n)
        assert np.array_equal(xg, xT)
        assert rel_err(mg, mT) <= 1e-12
        gt = torch.from_numpy(g).cuda()
        g0 = torch.empty_like(gt)
        dldD = mtpt.mtpt_adjoint_backward(h, gt, g0)
        # the handle is left in the final forward state
        assert np.array_equal(mtpt.mtpt_get_positions(h, 2, w.n), xT)
        dldD_again = mtpt.mtpt_adjoint_backward(h, gt, torch.empty_like(gt))
        assert dldD_again == dldD                          # deterministic
    finally:
        mtpt.mtpt_destroy(h)
    assert rel_err(g0.cpu().numpy(), lam) <= 1e-12
    # central finite differences of the oracle run in D (same normals)
    eps = 1e-5 * p.D
    runs = []
    for sgn in (+1, -1):
        opD = oracle_params(mtpt.Params(**{**p.__dict__, "D": p.D + sgn * eps}))
        _, x2, m2, pairs = _oracle_forward(opD, pos, mass, steps)
        L2, _, b2 = _loss_and_grad(w, x2, m2, target)
        runs.append((L2, b2, pairs))
    assert np.array_equal(runs[0][1], runs[1][1]), "a particle changed bin between +-eps"
    assert runs[0][2] == runs[1][2], "the pair set changed between +-eps"
    fd = (runs[0][0] - runs[1][0]) / (2 * eps)
    assert abs(dldD - fd) <= 1e-6 * max(abs(fd), 1e-3 * L), (dldD, fd)


def test_autograd_function_end_to_end():
    import torch
    from paper_2204_03756_gb300.autograd import binned_concentration, mtpt_run
    w, p, pos, mass, target, steps = _case(n=3000, steps=12)
    m0 = torch.from_numpy(mass).cuda().requires_grad_(True)
    D = torch.tensor(p.D, dtype=torch.float64, requires_grad=True)
    x0 = torch.from_numpy(pos).cuda()
    mT, xT = mtpt_run(m0, D, p, x0, steps, checkpoint_every=5)
    C = binned_concentration(xT, mT, w.lo, w.hi, NB)
    loss = ((C - torch.from_numpy(target).cuda()) ** 2).sum()
    loss.backward()
    # same gradients through the raw C ABI
    h = mtpt.mtpt_create(p)
    try:
        mtpt.mtpt_set_particles(h, 2, pos, mass)
        mtpt.mtpt_adjoint_forward(h, steps, 5)
        xg, mg = mtpt.mtpt_get_positions(h, 2, w.n), mtpt.mtpt_get_masses(h, w.n)
        _, g, _ = _loss_and_grad(w, xg, mg, target)
        gt = torch.from_numpy(g).cuda()
        g0 = torch.empty_like(gt)
        dldD = mtpt.mtpt_adjoint_backward(h, gt, g0)
    finally:
        mtpt.mtpt_destroy(h)
    assert rel_err(m0.grad.cpu().numpy(), g0.cpu().numpy()) <= 1e-12
    assert abs(D.grad.item() - dldD) <= 1e-10 * abs(dldD)


def test_adjoint_rejects_batches_and_missing_runs():
    import torch
    w, p, pos, mass, target, steps = _case(n=500, steps=2)
    h = mtpt.mtpt_create(p)
    try:
        mtpt.mtpt_set_particles(h, 2, pos, mass)
        g = torch.zeros(w.n, dtype=torch.float64, device="cuda")
        with pytest.raises(mtpt.MtptError) as e:
            mtpt.mtpt_adjoint_backward(h, g, torch.empty_like(g))
        assert e.value.code == mtpt.MTPT_ERR_STATE
    finally:
        mtpt.mtpt_destroy(h)
    b = mtpt.mtpt_create_batch([p, p])
    try:
        mtpt.mtpt_set_particles_batch(b, 2, [w.n, w.n], np.concatenate([pos, pos], 1),
                                      np.concatenate([mass, mass]))
        with pytest.raises(mtpt.MtptError):
            mtpt.mtpt_adjoint_forward(b, 2, 1)
    finally:
        mtpt.mtpt_destroy(b)
