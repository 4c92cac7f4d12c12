"""The warm start installed with pepo_set_warmstart_weights and applied inside
pepo_bp_converge equals the composed calls (features, forward, writer)."""
import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg
from oracle import mlp as om

pytestmark = pytest.mark.gpu


def test_integrated_warm_start_equals_the_composed_calls():
    import torch
    p = om.init_params(seed=4)
    flat = pkg.flat_params(p).astype(np.float32)
    base = dict(Lx=5, Ly=4, J=1.0, h=1.5, dt=0.05, order=2, obs=(2, 1), chi_max=10, precision="fp32")
    a = pkg.Engine(pkg.Config(warm_start=1, **base))
    a.set_warmstart_weights(torch.from_numpy(flat).cuda())
    b = pkg.Engine(pkg.Config(**base))
    net = pkg.Mlp(flat, max_rows=2 * b.num_bonds(0) * 10)
    for _ in range(4):
        a.trotter_step(1)
        b.trotter_step(1)
        b.ws_warm_start(net, gamma=0.25)
        sa, _ = a.bp_converge()
        sb, _ = b.bp_converge()
        Ca, _ = a.correlator()
        Cb, _ = b.correlator()
        assert list(sa) == list(sb)
        assert Ca[0] == Cb[0]
    a.close()
    b.close()


def test_weights_need_a_warm_start_instance():
    import torch
    e = pkg.Engine(pkg.Config(Lx=3, Ly=3, chi_max=4, precision="fp32"))
    n = int(e.lib.pepo_mlp_num_params())
    with pytest.raises(pkg.PepoError, match="warm_start"):
        e.set_warmstart_weights(torch.zeros(n, dtype=torch.float32, device="cuda"))
    e.close()
