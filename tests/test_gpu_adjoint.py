"""GPU parity of the discrete adjoint (lbm_lidar_misfit_grad) against the FP64 oracle's adjoint,
against central differences of the GPU forward model, and through torch.autograd.

The misfit is the lidar fit of the inflow (Sec. 3 boundary-condition paragraph, App. A): the
time-averaged horizontal wind at sampled fluid cells against a target, as a function of the level
speeds and the direction of the equilibrium inflow profile (App. D collision and streaming, D.1-D.11).
"""
import math

import numpy as np
import pytest

from oracle import adjoint as adj
from paper_2607_04516_b300 import synth

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3   # relative (max-norm) agreement of the FP32 gradient with the FP64 oracle / FD


def _small(faces, nz=8, nx=16, ny=12):
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[0:4, 4:7, 6:9] = 1
    solid[0:2, 8:10, 10:12] = 1
    cols = np.array([(3, 3), (12, 4), (4, 9)], np.int32)
    hts = np.array([1, 3, 5], np.int32)
    return solid, cols, hts


def _gpu_problem(solid, faces, cols, hts, target, T, n_avg, K, tau=0.55, cs=0.16):
    from paper_2607_04516_b300 import lbm
    dom = lbm.Domain(solid, faces, tau, cs, "f32")
    return lbm.LidarProblem(dom, cols, hts, target, T, n_avg, K)


CASES = [
    # faces, L, theta, T, n_avg, K
    (("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip"), 4, 0.4, 40, 12, 7),
    (("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip"), 3, 0.4, 30, 30, 30),
    (("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip"), 2, 0.0, 36, 10, 5),
    (("outflow", "inflow", "outflow", "inflow", "noslip", "outflow"), 4, math.pi + 0.5, 25, 25, 4),
]


@pytest.mark.parametrize("faces,L,theta,T,n_avg,K", CASES)
def test_gradient_matches_fp64_oracle_adjoint(faces, L, theta, T, n_avg, K):
    import torch
    solid, cols, hts = _small(faces)
    theta32 = float(np.float32(theta))
    rng = np.random.default_rng(L)
    truth = (0.05 + 0.01 * rng.random(L)).astype(np.float32)
    guess = (0.04 + 0.02 * rng.random(L)).astype(np.float32)
    p0 = adj.Problem(solid, faces, 0.55, 0.16, T, n_avg, cols, hts, np.zeros((3, 3, 2)), L)
    target = p0.forward(truth.astype(np.float64), theta32 + 0.05)[..., :2].astype(np.float32)
    prob = adj.Problem(solid, faces, 0.55, 0.16, T, n_avg, cols, hts, target.astype(np.float64), L)
    J_ref, ds_ref, dth_ref, _ = prob.gradient(guess.astype(np.float64), theta32)
    g_ref = np.concatenate([ds_ref, [dth_ref]])

    gp = _gpu_problem(solid, faces, cols, hts, target, T, n_avg, K)
    J, g, mean = gp.misfit_grad(guess, theta32)
    torch.cuda.synchronize()
    J, g = float(J), g.cpu().numpy()
    mean_ref = prob.forward(guess.astype(np.float64), theta32)
    np.testing.assert_allclose(mean.cpu().numpy()[..., :3], mean_ref, rtol=0, atol=1e-6)
    assert abs(J - J_ref) <= 1e-4 * J_ref
    err = np.abs(g - g_ref).max() / np.abs(g_ref).max()
    print(f"J {J:.6e} vs {J_ref:.6e}; gradient max rel err {err:.2e}")
    assert err <= TOL_GRAD


def test_gradient_matches_central_differences_of_the_gpu_forward():
    import torch
    faces = ("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip")
    solid, cols, hts = _small(faces)
    L, T, n_avg, K, theta = 4, 40, 16, 10, 0.4
    rng = np.random.default_rng(9)
    truth = (0.05 + 0.01 * rng.random(L)).astype(np.float32)
    guess = (truth * 0.85).astype(np.float32)
    gp = _gpu_problem(solid, faces, cols, hts, np.zeros((3, 3, 2), np.float32), T, n_avg, K)
    _, mean_t = gp.misfit(truth, theta + 0.05, target=False)
    target = mean_t[..., :2].float().contiguous()
    gp.target = target
    J, g, _ = gp.misfit_grad(guess, theta)
    g = g.cpu().numpy()
    h = 1e-3
    fd = []
    for l in range(L + 1):
        sp_p, sp_m = guess.astype(np.float64).copy(), guess.astype(np.float64).copy()
        th_p = th_m = theta
        if l < L:
            sp_p[l] += h
            sp_m[l] -= h
        else:
            th_p, th_m = theta + h, theta - h
        Jp, _ = gp.misfit(sp_p, th_p)
        Jm, _ = gp.misfit(sp_m, th_m)
        fd.append((float(Jp) - float(Jm)) / (2 * h))
    fd = np.array(fd)
    err = np.abs(g - fd).max() / np.abs(fd).max()
    print(f"gradient vs central differences (h = 1e-3): max rel err {err:.2e}")
    assert err <= TOL_GRAD


def test_autograd_function_returns_the_adjoint_gradient():
    import torch
    from paper_2607_04516_b300 import lbm
    faces = ("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip")
    solid, cols, hts = _small(faces)
    gp = _gpu_problem(solid, faces, cols, hts, np.full((3, 3, 2), 0.03, np.float32), 20, 5, 6)
    p = torch.tensor([0.04, 0.05, 0.045, 0.055, 0.3], dtype=torch.float64, requires_grad=True)
    J = lbm.lidar_misfit(p, gp)
    (2.0 * J).backward()
    J2, g2, _ = gp.misfit_grad(p.detach().numpy()[:-1], float(p.detach()[-1]))
    torch.cuda.synchronize()
    assert float(J.detach()) == float(J2)
    np.testing.assert_array_equal(p.grad.numpy(), 2.0 * g2.cpu().numpy())


def test_autograd_function_skips_the_reverse_sweep_without_a_gradient():
    """Under no_grad, or for a parameter tensor that needs no gradient, J comes from the forward
    model alone (no reverse sweep) and equals the differentiable evaluation's value."""
    import torch
    from paper_2607_04516_b300 import lbm
    faces = ("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip")
    solid, cols, hts = _small(faces)
    gp = _gpu_problem(solid, faces, cols, hts, np.full((3, 3, 2), 0.03, np.float32), 20, 5, 6)
    p = torch.tensor([0.04, 0.05, 0.045, 0.055, 0.3], dtype=torch.float64, requires_grad=True)
    J = lbm.lidar_misfit(p, gp)
    assert gp.reverse_sweeps == 1
    with torch.no_grad():
        J_ng = lbm.lidar_misfit(p, gp)
    J_nr = lbm.lidar_misfit(p.detach(), gp)
    torch.cuda.synchronize()
    assert gp.reverse_sweeps == 1
    assert not J_ng.requires_grad and not J_nr.requires_grad
    assert float(J_ng) == float(J.detach()) == float(J_nr)


def test_zero_misfit_gives_zero_gradient():
    import torch
    faces = ("inflow", "outflow", "periodic", "periodic", "noslip", "freeslip")
    solid, cols, hts = _small(faces)
    sp = np.array([0.05, 0.06], np.float32)
    gp = _gpu_problem(solid, faces, cols, hts, np.zeros((3, 3, 2), np.float32), 15, 6, 4)
    _, mean = gp.misfit(sp, 0.0, target=False)
    gp.target = mean[..., :2].float().contiguous()
    J, g, _ = gp.misfit_grad(sp, 0.0)
    torch.cuda.synchronize()
    # the target is the FP32-rounded mean: the residuals are at most half an FP32 ulp of |u|
    assert abs(float(J)) < 18 * (0.06 * 2.0 ** -24) ** 2
    assert np.abs(g.cpu().numpy()).max() < 1e-6   # residuals ~1e-9 times O(1) sensitivities


def test_rejects_non_fluid_samples_and_unsupported_domains():
    from paper_2607_04516_b300 import lbm
    faces = ("inflow", "outflow", "inflow", "outflow", "noslip", "freeslip")
    solid, cols, hts = _small(faces)
    bad = np.array([(7, 5)], np.int32)          # inside the first building at z = 1
    gp = _gpu_problem(solid, faces, bad, np.array([1], np.int32), np.zeros((1, 1, 2), np.float32), 5, 2, 2)
    with pytest.raises(lbm.LbmError):
        gp.misfit_grad(np.array([0.05], np.float32), 0.4)
    dom = lbm.Domain(solid, faces, 0.55, 0.16, "f16s")
    gp2 = lbm.LidarProblem(dom, cols, hts, np.zeros((3, 3, 2), np.float32), 5, 2, 2)
    with pytest.raises(lbm.LbmError):
        gp2.misfit_grad(np.array([0.05], np.float32), 0.4)


def test_assimilation_city_gradient_and_descent():
    """The 128 x 128 x 48 assimilation city (24 level speeds + direction, 8 lidar columns x 10
    heights, mean of the last 500 of 2000 steps, checkpoints every 100): the adjoint gradient
    against central differences (h = 1e-3) on six parameters, then gradient descent on the 25
    parameters lowers the misfit."""
    import torch
    from paper_2607_04516_b300 import lbm
    a = synth.assimilation_case()
    c = a.case
    dom = lbm.Domain(c.solid, c.faces, c.tau, c.cs, "f32")
    prob = lbm.LidarProblem(dom, a.cols, a.heights, np.zeros((8, 10, 2), np.float32), a.nsteps,
                            a.n_avg, a.checkpoint_every)
    _, mean = prob.misfit(a.speed_true.astype(np.float32), a.theta_true, target=False)
    prob.target = mean[..., :2].float().contiguous()
    p0 = np.concatenate([a.speed_guess, [a.theta_guess]])
    J0, g, _ = prob.misfit_grad(p0[:-1], p0[-1])
    J0, g = float(J0), g.cpu().numpy()
    h = 1e-3
    errs = []
    for l in (0, 5, 11, 17, 23, 24):
        pp, pm = p0.copy(), p0.copy()
        pp[l] += h
        pm[l] -= h
        Jp, _ = prob.misfit(pp[:-1], pp[-1])
        Jm, _ = prob.misfit(pm[:-1], pm[-1])
        fd = (float(Jp) - float(Jm)) / (2 * h)
        errs.append((l, g[l], fd))
    scale = max(abs(e[2]) for e in errs)
    worst = max(abs(e[1] - e[2]) for e in errs) / scale
    print("adjoint vs central differences (param, adjoint, fd):", errs, f"max rel err {worst:.2e}")
    assert worst <= TOL_GRAD
    # descent: steps along -g with a backtracking step length, 20 gradient evaluations
    p, J, step = p0.copy(), J0, 0.02
    for _ in range(20):
        Jc, gc, _ = prob.misfit_grad(p[:-1], p[-1])
        Jc, gc = float(Jc), gc.cpu().numpy()
        while step > 1e-6:
            q = p - step * gc / np.abs(gc).max()
            Jq, _ = prob.misfit(q[:-1], q[-1])
            if float(Jq) < Jc:
                p, J = q, float(Jq)
                step *= 1.5
                break
            step *= 0.5
    print(f"descent: J {J0:.3e} -> {J:.3e}; |speed - truth| {np.abs(p0[:-1] - a.speed_true).max():.2e} -> "
          f"{np.abs(p[:-1] - a.speed_true).max():.2e}; theta error {p0[-1] - a.theta_true:+.3f} -> "
          f"{p[-1] - a.theta_true:+.3f}")
    assert J < 0.5 * J0
