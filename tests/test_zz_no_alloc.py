"""pepo_set_site_static (allocation-free site upload) against pepo_set_site.

Two contexts receive the same seeded synthetic state; in the second, two
sites are uploaded back to back through the static staging buffer.  Every
site read back must be bit-identical between the two contexts, and a step of
the method from both states must give identical spectra.  Oversized and
wrongly typed uploads are rejected on the host.  The file name keeps it last
in collection order; it also passes on its own.
"""
import numpy as np
import pytest

import paper_2606_30985_gb300 as pkg

pytestmark = pytest.mark.gpu


def _engines_with_state(Lx, Ly, chi, precision="fp32"):
    from workloads.synthetic import bond_data, site_tensor
    cfg = pkg.Config(Lx=Lx, Ly=Ly, J=1.0, h=2.0, dt=0.05, order=2, obs=(1, 1), chi_max=chi,
                     precision=precision)
    bd = bond_data(Lx, Ly, chi)
    dt = np.float32 if precision != "fp64" else np.float64
    sites = [site_tensor(Lx, Ly, chi, 7, v, dt) for v in range(Lx * Ly)]
    a, b = pkg.Engine(cfg), pkg.Engine(cfg)
    for e in (a, b):
        e.set_bonds(0, bd["chi"], bd["lam"], bd["msgs"])
    return a, b, sites


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_static_upload_matches_set_site(precision):
    Lx, Ly, chi = 4, 4, 12
    a, b, sites = _engines_with_state(Lx, Ly, chi, precision)
    static_sites = (5, 6)                     # two interior sites, back to back
    for v, t in enumerate(sites):
        a.set_site(0, v, t)
        if v not in static_sites:
            b.set_site(0, v, t)
    for v in static_sites:
        b.set_site_static(0, v, sites[v])
    for v in range(Lx * Ly):
        ta, da = a.site(0, v)
        tb, db = b.site(0, v)
        assert da == db
        assert np.array_equal(ta, tb), v
    # the uploaded state evolves identically
    for e in (a, b):
        e.trotter_step(1)
    for bond in range(a.num_bonds(0)):
        assert np.array_equal(a.spectrum(0, bond), b.spectrum(0, bond)), bond
    a.close()
    b.close()


def test_static_upload_rejects_oversize_and_wrong_dtype():
    Lx, Ly, chi = 3, 3, 72                    # centre site: 4 * 72^4 floats = 107 MB > 16 MiB
    a, b, sites = _engines_with_state(Lx, Ly, chi)
    with pytest.raises(RuntimeError, match="static staging buffer holds"):
        b.set_site_static(0, 4, sites[4])
    with pytest.raises(RuntimeError, match="storage type"):
        b.set_site_static(0, 0, sites[0].astype(np.float64))
    b.set_site_static(0, 0, sites[0])          # a corner site fits
    a.set_site(0, 0, sites[0])
    assert np.array_equal(a.site(0, 0)[0], b.site(0, 0)[0])
    a.close()
    b.close()
