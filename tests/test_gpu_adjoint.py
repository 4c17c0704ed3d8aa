"""Hand-written adjoint of the coupled step against finite differences of the
FP64 oracle (central, FP64) and through the PyTorch autograd.Function.

Objective: L = (ubar - target)^2, ubar the mean rise velocity u_b,z over the
last `window` steps.  Gradients with respect to the drag scale, the bubble
diameter and the initial velocity field (along a seeded Gaussian direction).
Bar: 1e-4 relative for all three, against central differences of the FP64
oracle; a 16x16x32 column and a 32x32x64 column over 200 steps.
"""
import numpy as np
import pytest

from oracle import bubble as obub
from oracle import lattice as olat
from oracle.step import OracleSim
from paper_1710_07073_gb300 import lbm, workloads

pytestmark = pytest.mark.gpu

REL = 1e-4


def _problem(dims=(16, 16, 32), walls=olat.ALL_WALLS, positions=((8.0, 8.0, 6.0),), steps=60,
             every=10, window=20, g=1e-4, omega=1.6, target=0.0):
    from paper_1710_07073_gb300.adjoint import TerminalVelocityProblem
    return TerminalVelocityProblem(dims=dims, omega=omega, positions=np.array(positions),
                                   steps=steps, checkpoint_every=every, window=window,
                                   target=target, walls=walls, g=g)


def _oracle_loss(prob, drag_scale, diameter, u0):
    p = obub.BubbleParams(prob.omega, g=prob.g, drag_scale=drag_scale)
    sim = OracleSim(prob.dims, prob.omega, prob.walls, p)
    nx, ny, nz = prob.dims
    sim.set_fields(np.ones((nz, ny, nx)), u0)
    n = len(prob.positions)
    sim.set_bubbles(prob.positions, np.zeros((n, 3)), np.full(n, diameter))
    uz = []
    for _ in range(prob.steps):
        sim.step()
        uz.append(sim.u[:, 2].mean())
    ubar = np.mean(uz[-prob.window:])
    return (ubar - prob.target) ** 2


def _gpu_grads(prob, sd, d, u0):
    col = prob.column(sd, d, u0)
    loss = lbm.lbm_adj_forward(col.ctx, prob.steps, prob.checkpoint_every, prob.window,
                               prob.target)
    g_sd, g_d, g_u0 = lbm.lbm_adj_backward(col.ctx, 1.0, want_u0=True)
    col.close()
    return loss, g_sd, g_d.sum(), g_u0


def _check(prob, sd=1.0, d=2.5, eps=1.0, seed=4):
    P = workloads.gaussian_velocity_perturbation(prob.dims, seed=seed, amp=1e-4)
    loss, g_sd, g_d, g_u0 = _gpu_grads(prob, sd, d, eps * P)
    l_or = _oracle_loss(prob, sd, d, eps * P)
    assert abs(loss / l_or - 1.0) < 1e-4
    h = 1e-4
    fd_sd = (_oracle_loss(prob, sd + h, d, eps * P) - _oracle_loss(prob, sd - h, d, eps * P)) / (2 * h)
    fd_d = (_oracle_loss(prob, sd, d + h, eps * P) - _oracle_loss(prob, sd, d - h, eps * P)) / (2 * h)
    he = 1e-2
    fd_e = (_oracle_loss(prob, sd, d, (eps + he) * P) - _oracle_loss(prob, sd, d, (eps - he) * P)) / (2 * he)
    g_e = float((g_u0 * P.reshape(-1)).sum())
    print("drag scale: adjoint %.9e fd %.9e | diameter: adjoint %.9e fd %.9e | u0 dir: adjoint %.9e fd %.9e"
          % (g_sd, fd_sd, g_d, fd_d, g_e, fd_e))
    assert abs(g_sd / fd_sd - 1.0) < REL
    assert abs(g_d / fd_d - 1.0) < REL
    assert abs(g_e / fd_e - 1.0) < REL
    return g_u0


def test_adjoint_single_bubble_against_oracle_fd():
    _check(_problem())


def test_adjoint_mid_size_column_against_oracle_fd():
    # 32x32x64 over 200 steps with a checkpoint every 50 (the full-size
    # workload's segment length), d = 2.5.
    prob = _problem(dims=(32, 32, 64), positions=((16.0, 16.0, 8.0),), steps=200, every=50,
                    window=40)
    _check(prob, d=2.5)


def test_adjoint_two_bubbles_periodic_x_against_oracle_fd():
    # Two bubbles, a periodic x axis (window wraps), a partial last segment.
    prob = _problem(dims=(20, 16, 32), walls=olat.WALL_YM | olat.WALL_YP | olat.WALL_ZM | olat.WALL_ZP,
                    positions=((1.0, 8.0, 6.0), (12.0, 7.0, 9.0)), steps=47, every=9, window=15)
    _check(prob, d=2.0)


def test_autograd_function_matches_c_abi():
    import torch
    prob = _problem(steps=30, every=7, window=10)
    P = workloads.gaussian_velocity_perturbation(prob.dims, seed=4, amp=1e-4)
    sd = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    d = torch.tensor(2.5, dtype=torch.float64, requires_grad=True)
    eps = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    u0 = eps * torch.from_numpy(P)
    loss = prob.loss(sd, d, u0)
    loss.backward()
    ref_loss, g_sd, g_d, g_u0 = _gpu_grads(prob, 1.0, 2.5, P)
    assert abs(loss.item() - ref_loss) <= 1e-12 * abs(ref_loss)
    assert sd.grad.item() == pytest.approx(g_sd, rel=1e-12)
    assert d.grad.item() == pytest.approx(g_d, rel=1e-12)
    assert eps.grad.item() == pytest.approx(float((g_u0 * P.reshape(-1)).sum()), rel=1e-9)


def test_backward_needs_an_unchanged_forward_record():
    prob = _problem(steps=10, every=5, window=5)
    col = prob.column(1.0, 2.5, np.zeros((3,) + prob.dims[::-1]))
    lbm.lbm_adj_forward(col.ctx, 10, 5, 5, 0.0)
    lbm.lbm_step(col.ctx, 1)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_adj_backward(col.ctx)
    assert e.value.code == lbm.LBM_ERR_STATE


def test_adjoint_many_bubbles_against_oracle_fd():
    # Twelve bubbles with overlapping windows: a CTA per bubble for the
    # spreading adjoint and the sub-step reverse, the interpolation adjoints
    # added in bubble order, the drag-scale gradient summed in bubble order.
    rng = np.random.default_rng(12)
    pos = np.column_stack([rng.uniform(4.0, 12.0, 12), rng.uniform(4.0, 12.0, 12),
                           rng.uniform(5.0, 14.0, 12)])
    _check(_problem(positions=tuple(map(tuple, pos)), steps=40, every=10, window=10), d=2.0)


def test_adjoint_launch_count():
    # Every kernel of the forward record and of the reverse sweep is counted:
    # per step the coupled step's own launches (as lbm_step launches them from
    # the same state: the first steps after the bubbles are set or restored
    # take fewer) and the rise-velocity record; per checkpoint a bubble
    # snapshot; the final snapshot and the loss.  The reverse: per segment a
    # restore, its recomputed steps with two snapshots each; per reverse step
    # three adjoint kernels; the initial-field adjoint and the final restore.
    prob = _problem(steps=25, every=10, window=10)
    P = workloads.gaussian_velocity_perturbation(prob.dims, seed=4, amp=1e-4)

    def step_launches(k):
        col = prob.column(1.0, 2.5, P)
        n0 = lbm.lbm_launch_count(col.ctx)
        lbm.lbm_step(col.ctx, k)
        n = lbm.lbm_launch_count(col.ctx) - n0
        col.close()
        return n

    N, K = prob.steps, prob.checkpoint_every
    seg_lens = [min(K, N - s0) for s0 in range(0, N, K)]
    col = prob.column(1.0, 2.5, P)
    n0 = lbm.lbm_launch_count(col.ctx)
    lbm.lbm_adj_forward(col.ctx, N, K, prob.window, prob.target)
    n1 = lbm.lbm_launch_count(col.ctx)
    lbm.lbm_adj_backward(col.ctx, 1.0, want_u0=True)
    n2 = lbm.lbm_launch_count(col.ctx)
    col.close()
    assert n1 - n0 == step_launches(N) + N + len(seg_lens) + 2
    assert n2 - n1 == sum(1 + step_launches(L) + 2 * L for L in seg_lens) + 3 * N + 2
