"""Proposer and optimizer kernels against the FP64 oracle, and the gain of the
trained proposer over the plain optimizer (GPU).

Tolerances: the MLP runs in FP32 against an FP64 reference, so angles agree
to 1e-5 rad and gradients to 1e-4 of their largest entry; Adam agrees to
FP32/FP64 rounding.
"""

import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from oracle import reduced, statevector as sv
from paper_2402_02585_gb300 import _capi as C
from paper_2402_02585_gb300 import core, instances
from paper_2402_02585_gb300.optim import AngleOptimizer, canonicalize, single_angle_grid_start
from paper_2402_02585_gb300.proposer import Proposer

pytestmark = pytest.mark.gpu


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("dims,B", [((130, 256, 32), 300), ((10, 16, 6), 7), ((67, 100, 10), 129)])
def test_mlp_forward_backward_match_oracle(dims, B):
    rng = np.random.default_rng(B)
    params = instances.random_mlp_params(*dims, seed=B)
    params = (params + 0.02 * rng.standard_normal(params.shape)).astype(np.float32)
    x = rng.uniform(0, 1, (B, dims[0])).astype(np.float32)
    y = rng.uniform(0, 2 * np.pi, (B, dims[2])).astype(np.float32)
    P = torch.as_tensor(params).cuda()
    X = torch.as_tensor(x).cuda()
    Y = torch.as_tensor(y).cuda()
    ws = core.workspace(C.gqaoa_mlp_workspace_size(B, *dims))
    ang = torch.empty((B, dims[2]), dtype=torch.float32, device="cuda")
    C.gqaoa_mlp_forward(P.data_ptr(), *dims, X.data_ptr(), B, ang.data_ptr(), ws.data_ptr(),
                        ws.numel(), _stream())
    g = torch.empty_like(P)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    C.gqaoa_mlp_backward(P.data_ptr(), *dims, X.data_ptr(), Y.data_ptr(), B, g.data_ptr(),
                         loss.data_ptr(), ws.data_ptr(), ws.numel(), _stream())
    torch.cuda.synchronize()
    ref_ang, _ = omlp.forward(params.astype(np.float64), x.astype(np.float64), dims)
    ref_loss, ref_g = omlp.loss_and_grad(params.astype(np.float64), x.astype(np.float64),
                                         y.astype(np.float64), dims)
    assert np.max(np.abs(ang.cpu().numpy() - ref_ang)) < 1e-5
    assert abs(loss.item() - ref_loss) < 1e-5 * max(1.0, ref_loss)
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg - ref_g)) < 1e-4 * np.max(np.abs(ref_g))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_adam_matches_oracle(dtype):
    rng = np.random.default_rng(0)
    n = 1000
    p0 = rng.standard_normal(n)
    p = torch.as_tensor(p0, dtype=dtype).cuda()
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    rp, rm, rv = p0.copy(), np.zeros(n), np.zeros(n)
    fn = C.gqaoa_adam_f32 if dtype == torch.float32 else C.gqaoa_adam_f64
    for t in range(1, 6):
        g0 = rng.standard_normal(n)
        g = torch.as_tensor(g0, dtype=dtype).cuda()
        fn(p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr(), n, 0.01, 0.9, 0.999, 1e-8, t,
           1.0, _stream())
        rp, rm, rv = omlp.adam(rp, g0, rm, rv, t, 0.01)
    tol = 1e-5 if dtype == torch.float32 else 1e-12
    assert np.max(np.abs(p.cpu().numpy() - rp)) < tol


def test_features_match_oracle():
    prop = Proposer(p=4)
    hists, ns, ms = [], [], []
    for i, n in enumerate([8, 10, 12]):
        m = 4 * n
        hists.append(sv.histogram(instances.random_3sat(n, m, i), n))
        ns.append(n)
        ms.append(m)
    x = prop.features(hists, ns, ms).cpu().numpy()
    for i in range(3):
        ref = omlp.features(hists[i], ns[i], ms[i], 130)
        assert np.allclose(x[i], ref, atol=1e-7, rtol=1e-6)


def test_angle_optimizer_improves_and_matches_reduced_model():
    n, m, p, B = 12, 50, 4, 6
    costs, hists = [], []
    for i in range(B):
        c, h = core.build_cost(instances.random_3sat(n, m, 500 + i), n)
        costs.append(c)
        hists.append(h.cpu().numpy())
    opt = AngleOptimizer(torch.stack(costs), n, m, p)
    g0 = np.stack([instances.random_angles(p, 600 + i)[0] for i in range(B)])
    b0 = np.stack([instances.random_angles(p, 600 + i)[1] for i in range(B)])
    opt.reset(g0, b0)
    v0 = opt.evaluate().cpu().numpy()
    for i in range(B):
        assert abs(v0[i] - reduced.grad(hists[i], g0[i], b0[i])[0]) < 1e-6
    res = opt.run(60, lr=0.05)
    vals = res["values"]
    assert np.all(vals[-1] >= vals[0] - 1e-9)
    assert np.mean(vals[-1]) > 1.5 * np.mean(vals[0])
    g, b = opt.angles()
    for i in range(B):
        ref = reduced.objective_value(hists[i], g[i].cpu().numpy(), b[i].cpu().numpy())
        assert abs(vals[-1][i] - ref) < 1e-6


def test_single_angle_grid_start_is_grid_argmax():
    n, m, p = 10, 42, 3
    cost, hist = core.build_cost(instances.random_3sat(n, m, 0), n)
    g, b = single_angle_grid_start(cost[None], n, m, p, grid=8)
    h = hist.cpu().numpy()
    best = max(((reduced.objective_value(h, [gg] * p, [bb] * p), gg, bb)
                for gg in (np.arange(8) + 0.5) * np.pi / 4
                for bb in (np.arange(8) + 0.5) * np.pi / 8))
    assert abs(reduced.objective_value(h, [g[0]] * p, [b[0]] * p) - best[0]) < 1e-6


def test_canonicalize_preserves_objective():
    h = sv.histogram(instances.random_3sat(9, 38, 1), 9)
    rng = np.random.default_rng(2)
    G = rng.uniform(-7, 7, (5, 3))
    Bt = rng.uniform(-7, 7, (5, 3))
    lab = canonicalize(G, Bt)
    assert np.all(lab >= 0) and np.all(lab < 2 * np.pi) and np.all(lab[:, 0] <= np.pi)
    for i in range(5):
        assert abs(reduced.objective_value(h, G[i], Bt[i])
                   - reduced.objective_value(h, lab[i, :3], lab[i, 3:])) < 1e-12


def test_trained_proposer_gains_over_plain_optimizer():
    """Train on optimizer-produced labels for small instances, then start the
    plain optimizer from the proposal on larger held-out instances: it must
    reach 95 % of the plain (random-start) optimizer's final P in fewer steps."""
    from paper_2402_02585_gb300 import study
    p = 4
    train = study.make_instances(240, seed=1, n_values=range(8, 13), d_lo=3.0, d_hi=5.0)
    X, Y = study.generate_labels(train, p=p, grid=12, steps=150, lr=0.05)
    prop = Proposer(p=p, d_h=64, seed=0)
    losses = prop.fit(X, Y, epochs=150, batch=64, lr=1e-3)
    assert losses[-1] < 0.2 * losses[0]
    test = study.make_instances(32, seed=2, n_values=[14], d_lo=3.0, d_hi=5.0)
    ev = study.evaluate(prop, test, p=p, plain_steps=200, max_steps=200, lr=0.05, seed=5)
    print(ev)
    assert ev["hit_rate"] >= 0.9
    assert ev["median_steps_proposer"] < ev["median_steps_plain"]
    assert ev["median_wall_proposer"] < ev["median_wall_plain"]


def test_proposer_state_roundtrip_and_optimizer_resume(tmp_path):
    prop = Proposer(p=3, d_h=32, seed=4)
    x = torch.rand((5, 130), device="cuda")
    a0 = prop.predict(x).clone()
    torch.save(prop.state_dict(), tmp_path / "prop.pt")
    other = Proposer(p=3, d_h=32, seed=99)
    other.load_state_dict(torch.load(tmp_path / "prop.pt"))
    assert torch.equal(other.predict(x), a0)
    # the optimizer resumes from saved angles: same values from the same angles
    n, m, p = 11, 46, 3
    cost = torch.stack([core.build_cost(instances.random_3sat(n, m, 40 + i), n)[0] for i in range(2)])
    opt = AngleOptimizer(cost, n, m, p)
    opt.reset(np.full((2, p), 0.4), np.full((2, p), 2.0))
    opt.run(10)
    g, b = opt.angles()
    np.save(tmp_path / "angles.npy", torch.stack([g, b]).cpu().numpy())
    v_before = opt.evaluate().clone()
    saved = np.load(tmp_path / "angles.npy")
    opt2 = AngleOptimizer(cost, n, m, p)
    opt2.reset(saved[0], saved[1])
    assert torch.equal(opt2.evaluate(), v_before)
