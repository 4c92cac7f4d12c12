"""Learned BP warm start on the GPU against the oracle (oracle/mlp.py).

Kernels checked one by one: the BF16 forward pass, the gradient of the mean
squared error (the GPU backward against the oracle's backward evaluated at the
same BF16 rounding points), one Adam update, the feature rows of an evolved
state, the target log-diagonals and the message writer.
"""
import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg
from oracle import mlp as om

pytestmark = pytest.mark.gpu


def _rand_case(rows=300, seed=11):
    rng = np.random.default_rng(seed)
    p = om.init_params(seed=seed)
    for k in p:
        p[k] = p[k] + 0.02 * rng.standard_normal(p[k].shape)
    X = rng.standard_normal((rows, om.NF)).astype(np.float32)
    t = rng.standard_normal(rows).astype(np.float32)
    return p, X, t


def _rnd(a):
    return om.bf16(a).astype(np.float64)


def test_forward_and_gradient_match_oracle():
    import torch
    p, X, t = _rand_case()
    net = pkg.Mlp(pkg.flat_params(p), max_rows=1024)
    Xd = torch.from_numpy(X).cuda()
    td = torch.from_numpy(t).cuda()
    y = net.forward(Xd).cpu().numpy()
    p32 = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}   # the GPU's FP32 master copy
    yr, cache = om.forward(p32, X.astype(np.float64), rnd=_rnd)
    assert np.max(np.abs(y - yr)) <= 2e-3 * max(1.0, np.max(np.abs(yr)))
    loss, g = net.gradient(Xd, td, want_grad=True)
    gr = om.backward(p32, cache, yr, t.astype(np.float64), rnd=_rnd)
    assert abs(loss - om.loss(yr, t)) <= 1e-3 * om.loss(yr, t)
    G = pkg.unflat_params(g)
    for k in gr:
        ref = gr[k].reshape(-1)
        got = G[k].reshape(-1)
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err < 1e-2, (k, err)
        # element by element: both sides round to BF16 at the same points, so
        # an entry differs by the FP32 accumulation order and by an occasional
        # BF16 rounding that falls the other way (2^-8 of the entry's largest
        # contributions): bounded by 2^-7 of the entry plus 2^-7 of the tensor's scale
        bound = 2.0 ** -7 * (np.abs(ref) + np.max(np.abs(ref)))
        worst = int(np.argmax(np.abs(got - ref) - bound))
        assert np.all(np.abs(got - ref) <= bound), (k, worst, got[worst], ref[worst])


def test_adam_step_matches_oracle():
    import torch
    p, X, t = _rand_case(rows=200, seed=3)
    net = pkg.Mlp(pkg.flat_params(p), max_rows=256)
    loss, g = net.gradient(torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda(), want_grad=True)
    net.adam_step(1e-3)
    got = net.params()
    ref = {k: v.astype(np.float32).astype(np.float64) for k, v in p.items()}
    opt = om.Adam(ref, lr=1e-3)
    opt.step(ref, pkg.unflat_params(g))
    assert np.max(np.abs(got - pkg.flat_params(ref))) < 1e-6


def test_features_targets_and_apply_on_an_evolved_state():
    import torch
    cfg = pkg.Config(Lx=4, Ly=3, J=1.0, h=1.5, dt=0.05, order=2, obs=(1, 1), chi_max=6, precision="fp32")
    eng = pkg.Engine(cfg)
    eng.trotter_step(6)
    eng.bp_converge()
    nb = eng.num_bonds(0)
    lam = np.zeros((nb, cfg.chi_max))
    chi = np.zeros(nb, dtype=int)
    for b in range(nb):
        s = eng.spectrum(0, b)
        chi[b] = len(s)
        lam[b, :len(s)] = s
    X = eng.ws_features().cpu().numpy()
    Xr, idx = om.features(4, 3, (1, 1), chi, lam, step=6, dt=0.05, h=1.5, J=1.0)
    assert X.shape == Xr.shape
    assert np.max(np.abs(X - Xr)) < 1e-5
    t = eng.ws_targets().cpu().numpy()
    for r, (b, d, k) in enumerate(idx):
        M = eng.message(0, b, d)
        assert abs(t[r] - np.log(max(M[k, k], 1e-300))) < 1e-5
    y = torch.linspace(-1.0, 1.0, X.shape[0], device="cuda", dtype=torch.float32)
    yh = y.cpu().numpy()
    before = {(b, d): np.diag(eng.message(0, b, d)).copy() for b in range(nb) for d in range(2)}
    eng.ws_apply(y, gamma=0.25)
    for b in range(nb):
        for d in range(2):
            rows = [r for r in range(len(idx)) if idx[r][0] == b and idx[r][1] == d]
            M = eng.message(0, b, d)
            ref = om.warm_message(yh[rows].astype(np.float64), plain_diag=before[(b, d)], gamma=0.25)
            assert M.shape == ref.shape and np.max(np.abs(M - ref)) < 1e-6
    eng.ws_apply(y, gamma=1.0)
    for b in range(nb):
        for d in range(2):
            rows = [r for r in range(len(idx)) if idx[r][0] == b and idx[r][1] == d]
            ref = om.warm_message(yh[rows].astype(np.float64))
            assert np.max(np.abs(eng.message(0, b, d) - ref)) < 1e-6
    eng.close()


def _trajectory(h, obs, steps, net=None, gamma=pkg.WS_GAMMA, collect=None):
    cfg = pkg.Config(Lx=6, Ly=6, J=1.0, h=h, dt=0.05, order=2, obs=obs, chi_max=12, precision="fp32")
    eng = pkg.Engine(cfg)
    sweeps, Cs = [], []
    for _ in range(steps):
        eng.trotter_step(1)
        X = eng.ws_features().clone()
        if net is not None:
            eng.ws_apply(net.forward(X), gamma=gamma)
        sw, _ = eng.bp_converge()
        C, _ = eng.correlator()
        sweeps.append(sw[0])
        Cs.append(C[0])
        if collect is not None:
            collect.append((X, eng.ws_targets().clone()))
    eng.close()
    return sweeps, Cs


def test_trained_network_saves_bp_sweeps():
    """Train on two 6x6 trajectories (the GPU's own forward / backward / Adam
    kernels), then run a held-out trajectory (other h, other observable site)
    with and without the warm start: fewer total BP sweeps, same C(t)."""
    import torch
    data = []
    for h, obs in ((1.5, (2, 2)), (2.5, (3, 2))):
        _trajectory(h, obs, 20, collect=data)
    X = torch.cat([d[0] for d in data])
    T = torch.cat([d[1] for d in data])
    net = pkg.Mlp(pkg.flat_params(om.init_params(seed=0)), max_rows=4096)
    g = torch.Generator(device="cuda").manual_seed(0)
    first = None
    for it in range(1500):
        idx = torch.randint(0, X.shape[0], (4096,), device="cuda", generator=g)
        loss, _ = net.gradient(X[idx], T[idx])
        first = loss if first is None else first
        net.adam_step(1e-3)
    assert loss < 1e-2 * first
    plain, Cp = _trajectory(2.0, (3, 3), 20)
    warm, Cw = _trajectory(2.0, (3, 3), 20, net=net)
    print("BP sweeps over 20 held-out steps: plain %d, warm start %d (%s vs %s)" % (sum(plain), sum(warm), plain, warm))
    assert sum(warm) < sum(plain)
    assert max(abs(a - b) for a, b in zip(Cp, Cw)) < 1e-3
