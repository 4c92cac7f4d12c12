"""Argument checks of the ctypes binding that need no GPU: device buffers are
validated before their raw pointer reaches the library."""
import pytest
import torch

import paper_2606_30985_gb300 as pkg


def test_device_tensor_rejects_host_wrong_dtype_short_and_strided():
    with pytest.raises(pkg.PepoError, match="GPU"):
        pkg._device_tensor(torch.zeros(16, dtype=torch.uint8), torch.uint8, 8, "save_state")
    with pytest.raises(pkg.PepoError, match="torch tensor"):
        pkg._device_tensor(b"\x00" * 16, torch.uint8, 8, "save_state")


@pytest.mark.gpu
def test_device_tensor_checks_on_cuda():
    t = torch.zeros(16, dtype=torch.uint8, device="cuda")
    assert pkg._device_tensor(t, torch.uint8, 16, "x") is t
    with pytest.raises(pkg.PepoError, match="dtype"):
        pkg._device_tensor(t, torch.float32, 1, "x")
    with pytest.raises(pkg.PepoError, match="at least"):
        pkg._device_tensor(t, torch.uint8, 17, "x")
    with pytest.raises(pkg.PepoError, match="contiguous"):
        pkg._device_tensor(torch.zeros(4, 4, dtype=torch.uint8, device="cuda").t(), torch.uint8, 1, "x")


@pytest.mark.parametrize("Lx,Ly,obs", [(4, 3, (2, 1)), (5, 5, None), (1, 6, (0, 2)), (7, 2, (6, 0))])
def test_spatial_observables_match_the_oracle_formulas(Lx, Ly, obs):
    # the binding's R_L1, R_L2, S_frac of a weight map (host arithmetic, no
    # GPU) against the oracle's restatement of Appendix A.3
    import numpy as np
    from oracle import bp as obp
    cfg = pkg.Config(Lx=Lx, Ly=Ly, obs=obs)
    rng = np.random.default_rng(Lx * 10 + Ly)
    n = rng.random((Ly, Lx)) ** 3
    n[rng.random((Ly, Lx)) < 0.3] = 0.0
    got = pkg.spatial_observables(n, cfg)
    o = obs if obs is not None else ((Lx - 1) // 2, (Ly - 1) // 2)
    want = obp.spatial_observables(n.reshape(-1), Lx, Ly, o)
    for k in ("R_L1", "R_L2", "S_frac"):
        assert abs(got[k] - want[k]) < 1e-12, k
    zero = pkg.spatial_observables(np.zeros((Ly, Lx)), cfg)
    assert zero["R_L1"] == zero["R_L2"] == zero["S_frac"] == 0.0


def test_difference_field():
    import numpy as np
    rng = np.random.default_rng(3)
    base = rng.random((5, 5))
    sym = sum(np.rot90(base, k) for k in range(4))        # C4-symmetric about the centre
    other = sym * 0.9 + 0.05
    d = pkg.difference_field(sym, other)
    assert np.allclose(d["dn"], sym - other)
    assert abs(d["max_abs"] - np.max(np.abs(sym - other))) < 1e-15
    assert d["c4_asym"] < 1e-12
    skew = other.copy()
    skew[0, 1] += 1e-3
    assert abs(pkg.difference_field(sym, skew)["c4_asym"] - 1e-3) < 1e-12
    assert "c4_asym" not in pkg.difference_field(np.zeros((3, 4)), np.ones((3, 4)))
    with pytest.raises(pkg.PepoError):
        pkg.difference_field(np.zeros((3, 3)), np.zeros((3, 4)))
