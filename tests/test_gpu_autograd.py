"""The differentiable lattice transform: gradient of ||reconstruct(y) - c||^2
against central finite differences and against the oracle's dense R^H."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1711_05152_gb300 as P
import workloads as W
from oracle import lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    P.lib()


def _loss_and_grad(plan, y, c):
    from paper_1711_05152_gb300 import autograd as AG
    y = y.clone().requires_grad_(True)
    loss = (AG.reconstruct(y, plan) - c).abs().pow(2).sum()
    loss.backward()
    return loss.detach(), y.grad


def _fd_check(plan, y, c, ndir, h=1e-6, seed=0):
    _, g = _loss_and_grad(plan, y, c)
    gen = torch.Generator(device=y.device).manual_seed(seed)
    worst = 0.0
    for _ in range(ndir):
        v = torch.complex(torch.randn(y.shape, generator=gen, device=y.device, dtype=torch.float64),
                          torch.randn(y.shape, generator=gen, device=y.device, dtype=torch.float64))
        # direction scaled to |y|: the step h is relative to the point (the loss
        # is exactly quadratic, so central differences carry only rounding)
        v = v * (y.abs().pow(2).sum().sqrt() / v.abs().pow(2).sum().sqrt())
        # (L(y + h v) - L(y - h v)) / 2h, with the difference taken entry by entry
        # (|r+|^2 - |r-|^2 = Re((r+ - r-) conj(r+ + r-))) before the sum, so the
        # rounding of two large sums does not swamp it
        rp = plan.reconstruct(y + h * v) - c
        rm = plan.reconstruct(y - h * v) - c
        fd = float(torch.real((rp - rm) * torch.conj(rp + rm)).sum()) / (2 * h)
        an = float(torch.real(torch.vdot(g.reshape(-1), v.reshape(-1))))
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-30))
    return worst


def test_gradient_finite_differences_small():
    rng = np.random.default_rng(0)
    I, _ = W.diff_problem(500, 4, 8, 1, seed=1)
    pl = P.plan_search(I, seed=2)
    y = torch.from_numpy(W.complex_normal(rng, (2, pl.sum_M))).cuda()
    c = torch.from_numpy(W.complex_normal(rng, (2, pl.nI))).cuda()
    assert _fd_check(pl, y, c, ndir=6) < 1e-6


def test_gradient_matches_dense_transpose_2000():
    """2000-frequency subset of the [-64, 64]^20 problem, its own lattice; the
    gradient 2 R^H (R y - c) against the oracle's entry-by-entry matrix R."""
    I, rng = W.diff_problem(100_000, 20, 64, 64, seed=4)
    sub = I[np.sort(np.random.default_rng(5).choice(I.shape[0], 2000, replace=False))].astype(np.int64)
    pl = P.plan_search(sub, seed=6)
    ml = lattice.search(sub, seed=6, t=20)
    assert list(pl.M) == ml.M
    yh = W.complex_normal(rng, (2, pl.sum_M))
    ch = W.complex_normal(rng, (2, 2000))
    _, g = _loss_and_grad(pl, torch.from_numpy(yh).cuda(), torch.from_numpy(ch).cuda())
    g = g.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(ml.M)])
    inv_cnt = 1.0 / np.maximum(ml.counter(), 1)
    # R = [R_1 .. R_L] column blocks, R_l[k, j] = [k in I_l] / (counter_k M_l) e^{-2 pi i j k.z_l / M_l}
    blocks = [lattice.dense_reconstruct_matrix(sub, lattice.MultiLattice([M], [z], [IL], True, 1))
              * inv_cnt[:, None] for M, z, IL in zip(ml.M, ml.z, ml.unique)]
    for h in range(2):
        resid = sum(B @ yh[h, offs[l]:offs[l + 1]] for l, B in enumerate(blocks)) - ch[h]
        want = np.concatenate([2.0 * (B.conj().T @ resid) for B in blocks])
        err = np.max(np.abs(g[h] - want)) / np.max(np.abs(want))
        assert err < 1e-10, err


@pytest.mark.slow
def test_gradient_finite_differences_full_size():
    """10^5 frequencies in [-64, 64]^20, its Algorithm 1 lattice, 64
    right-hand sides; target c = R(y0) + noise; central differences with
    step 1e-6 along random directions."""
    I, rng = W.diff_problem(100_000, 20, 64, 64, seed=4)
    pl = P.plan_search(I, seed=7)
    assert pl.n_uncovered == 0
    y0 = torch.from_numpy(W.complex_normal(rng, (64, pl.sum_M))).cuda()
    c = pl.reconstruct(y0) + 0.01 * torch.from_numpy(W.complex_normal(rng, (64, pl.nI))).cuda()
    y = torch.from_numpy(W.complex_normal(rng, (64, pl.sum_M))).cuda()
    assert _fd_check(pl, y, c, ndir=4) < 1e-6
