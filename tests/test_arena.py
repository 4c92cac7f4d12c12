"""Arena sizing (pepo_required_bytes) is host logic: checked without a GPU."""
import paper_2606_30985_gb300 as pkg


def _bytes(cfgs):
    lib = pkg.load_library()
    return int(lib.pepo_required_bytes(pkg._cfg_array(cfgs), len(cfgs)))


def test_warm_start_workspace_is_carved_only_when_asked_for():
    base = dict(Lx=6, Ly=5, chi_max=24, precision="tf32x3")
    plain = _bytes([pkg.Config(**base)])
    ws = _bytes([pkg.Config(warm_start=1, **base)])
    lib = pkg.load_library()
    nb = 6 * 4 + 5 * 5                          # horizontal + vertical bonds of 6x5
    rows = 2 * nb * 24
    want = lib.pepo_mlp_required_bytes(rows) - 256 + rows * (pkg.WS_FEATURES + 1) * 4
    assert want <= ws - plain <= want + 4 * 256   # plus alignment of three carved blocks
    # sized for the largest warm-started instance of a batch; plain instances add nothing
    mixed = _bytes([pkg.Config(warm_start=1, **base), pkg.Config(Lx=3, Ly=3, chi_max=8, precision="tf32x3")])
    both = _bytes([pkg.Config(**base), pkg.Config(Lx=3, Ly=3, chi_max=8, precision="tf32x3")])
    assert want <= mixed - both <= want + 4 * 256


def test_invalid_configuration_needs_no_arena():
    assert _bytes([pkg.Config(Lx=1, Ly=1)]) == 0
    assert _bytes([pkg.Config(chi_max=129)]) == 0
