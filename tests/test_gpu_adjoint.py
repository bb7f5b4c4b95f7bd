"""Hand-written adjoint (sph_record / sph_backward behind a torch.autograd
Function) vs the FP64 oracle's dual-number directional derivatives, which
the CPU tests pin to central differences (marked gpu).

Loss: L = mean over fluid particles of |x_i(T) - target_i|^2 (minimum
image), target = initial positions + seeded N(0, (0.1 dp)^2); dt frozen.
Tolerance: |g.v - J(v)| <= 1e-3 max(|J(v)|, rms_v |J|) for seeded unit
directions v in u0 space, and the same for d/dalpha.
"""
import multiprocessing as mp

import numpy as np
import pytest

import oracle
from paper_2207_11328_gb300 import scenes
from tests.gpu_common import oracle_jvp_task, oracle_params_kw, require_gpu, sim_for

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _loss_torch(x_T, tgt, L, fluid):
    import torch
    d = x_T - tgt
    for a in range(3):
        if L[a] is not None:
            d[:, a] = d[:, a] - L[a] * torch.round(d[:, a] / L[a])
    return (d[fluid] ** 2).sum() / int(fluid.sum())


def _gpu_grad(s, tgt, T, K, alpha):
    import torch
    from paper_2207_11328_gb300.autograd import rollout
    dev = torch.device("cuda", 0)
    sim = sim_for(s)
    u0 = torch.tensor(s.vel, dtype=torch.float32, device=dev, requires_grad=True)
    al = torch.tensor(alpha, dtype=torch.float64, requires_grad=True)
    x_T = rollout(u0, al, sim, torch.tensor(s.pos, device=dev), torch.tensor(s.delta), torch.tensor(s.mass),
                  torch.tensor(s.ptype), T=T, K=K)
    Ls = [s.size[a] if (s.periodic >> a) & 1 else None for a in range(3)]
    fluid = torch.tensor(s.ptype == 0, device=dev)
    L = _loss_torch(x_T, torch.tensor(tgt, device=dev), Ls, fluid)
    L.backward()
    return float(L), u0.grad.double().cpu().numpy(), float(al.grad), sim


def _check(g, ga, J, Ja, dirs, what):
    gv = np.array([np.sum(g * v.reshape(-1, 3)) for v in dirs])
    scale = np.maximum(np.abs(J), np.sqrt(np.mean(J ** 2)))
    rel = np.abs(gv - J) / scale
    print(f"{what}: max rel err over {len(dirs)} directions {rel.max():.2e}; alpha {abs(ga - Ja) / abs(Ja):.2e}")
    assert np.all(rel <= TOL), rel
    assert abs(ga - Ja) <= TOL * abs(Ja)


def _box(n, dt=3.9e-4):
    s = scenes.periodic_box(n_per_axis=n)
    s.dt_fixed = dt
    tgt = s.pos + scenes.seeded_normal(s.pos.shape, 0.1 * s.dp, 2207_11331)
    return s, tgt


def test_adjoint_small_box_vs_oracle():
    s, tgt = _box(8)
    T, K = 8, 4
    L, g, ga, sim = _gpu_grad(s, tgt, T, K, s.alpha)
    p = oracle.params(s)
    L_ora, _ = oracle.loss_jvp(p, s.pos, s.vel, s.delta, s.mass, s.ptype, T, s.dt_fixed, tgt)
    assert L == pytest.approx(L_ora, rel=1e-5)
    dirs = scenes.seeded_directions(3 * s.n, 16)
    J = np.array([oracle.loss_jvp(p, s.pos, s.vel, s.delta, s.mass, s.ptype, T, s.dt_fixed, tgt,
                                  v.reshape(-1, 3))[1] for v in dirs])
    Ja = oracle.loss_jvp(p, s.pos, s.vel, s.delta, s.mass, s.ptype, T, s.dt_fixed, tgt, None, 1.0)[1]
    _check(g, ga, J, Ja, dirs, "box 8^3 T=8")


def test_adjoint_deterministic_and_checkpoint_invariant():
    s, tgt = _box(8)
    ref = None
    for K in (8, 4, 2, 1):
        L, g, ga, _ = _gpu_grad(s, tgt, 8, K, s.alpha)
        if ref is None:
            ref = (L, g, ga)
        else:
            assert L == ref[0] and np.array_equal(g, ref[1]) and ga == ref[2]


def test_adjoint_dam_with_boundaries_vs_oracle():
    s = scenes.dam_break(dp=0.05)
    s.dt_fixed = 4e-4
    tgt = s.pos + scenes.seeded_normal(s.pos.shape, 0.1 * s.dp, 2207_11332)
    T, K = 6, 3
    L, g, ga, _ = _gpu_grad(s, tgt, T, K, s.alpha)
    assert np.all(g[s.ptype == 1] == 0)
    p = oracle.params(s)
    dirs = scenes.seeded_directions(3 * s.n, 8, seed=5)
    for v in dirs:   # directions in the fluid's velocities only (boundary velocities are constants)
        v.reshape(-1, 3)[s.ptype == 1] = 0
    J = np.array([oracle.loss_jvp(p, s.pos, s.vel, s.delta, s.mass, s.ptype, T, s.dt_fixed, tgt,
                                  v.reshape(-1, 3))[1] for v in dirs])
    Ja = oracle.loss_jvp(p, s.pos, s.vel, s.delta, s.mass, s.ptype, T, s.dt_fixed, tgt, None, 1.0)[1]
    _check(g, ga, J, Ja, dirs, "dam dp=0.05 T=6")


def test_adjoint_32cube_T64_64_directions():
    # 32^3 periodic box, same physics as the 16^3 box, T = 64, checkpoint every 8
    s, tgt = _box(32)
    T, K = 64, 8
    dirs = scenes.seeded_directions(3 * s.n, 64)
    pkw = oracle_params_kw(s)
    args = [(pkw, s.pos, s.vel, s.delta, s.mass, s.ptype, T, s.dt_fixed, tgt, v.reshape(-1, 3), 0.0) for v in dirs]
    args.append((pkw, s.pos, s.vel, s.delta, s.mass, s.ptype, T, s.dt_fixed, tgt, None, 1.0))
    eps = 1e-4
    fd_dirs = dirs[:2]
    for v in fd_dirs:
        for sg in (1.0, -1.0):
            args.append((pkw, s.pos, s.vel + sg * eps * v.reshape(-1, 3), s.delta, s.mass, s.ptype, T, s.dt_fixed,
                         tgt, None, 0.0))
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, mp.cpu_count())) as pool:
        res = pool.map_async(oracle_jvp_task, args)
        L, g, ga, _ = _gpu_grad(s, tgt, T, K, s.alpha)
        out = res.get(timeout=3000)
    J = np.array([o[1] for o in out[:64]])
    Ja = out[64][1]
    assert L == pytest.approx(out[0][0], rel=1e-5)
    _check(g, ga, J, Ja, dirs, "box 32^3 T=64")
    fd = [(out[65 + 2 * k][0] - out[66 + 2 * k][0]) / (2 * eps) for k in range(len(fd_dirs))]
    for k, v in enumerate(fd_dirs):
        gv = float(np.sum(g * v.reshape(-1, 3)))
        assert abs(gv - fd[k]) <= TOL * max(abs(fd[k]), np.sqrt(np.mean(J ** 2))), (gv, fd[k])


def test_rollout_refuses_a_replaced_recording():
    # two rollouts on one context: the second forward replaces the first's tape, so the
    # first's backward must refuse instead of returning the second trajectory's gradients;
    # the second's own backward still works and matches a fresh context's gradient
    import torch
    from paper_2207_11328_gb300.autograd import rollout
    s, tgt = _box(8)
    dev = torch.device("cuda", 0)
    sim = sim_for(s)
    args = (sim, torch.tensor(s.pos, device=dev), torch.tensor(s.delta), torch.tensor(s.mass), torch.tensor(s.ptype))
    u_a = torch.tensor(s.vel, dtype=torch.float32, device=dev, requires_grad=True)
    u_b = torch.tensor(s.vel, dtype=torch.float32, device=dev, requires_grad=True)
    al = torch.tensor(s.alpha, dtype=torch.float64, requires_grad=True)
    g0 = sim.tape_generation()
    x_a = rollout(u_a, al, *args, T=4, K=2)
    g1 = sim.tape_generation()
    x_b = rollout(u_b, al, *args, T=4, K=2)
    g2 = sim.tape_generation()
    assert g1 > g0 and g2 > g1
    with pytest.raises(RuntimeError, match="replaced"):
        x_a.sum().backward()
    x_b.sum().backward()
    _, g_ref, _, _ = _gpu_grad_sum(s, T=4, K=2)
    assert np.array_equal(u_b.grad.cpu().numpy(), g_ref)


def _gpu_grad_sum(s, T, K):
    import torch
    from paper_2207_11328_gb300.autograd import rollout
    dev = torch.device("cuda", 0)
    sim = sim_for(s)
    u0 = torch.tensor(s.vel, dtype=torch.float32, device=dev, requires_grad=True)
    al = torch.tensor(s.alpha, dtype=torch.float64, requires_grad=True)
    x = rollout(u0, al, sim, torch.tensor(s.pos, device=dev), torch.tensor(s.delta), torch.tensor(s.mass),
                torch.tensor(s.ptype), T=T, K=K)
    x.sum().backward()
    return None, u0.grad.cpu().numpy(), float(al.grad), sim
