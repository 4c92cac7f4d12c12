"""Autotuner cache lookup (host logic only; the sweep itself runs on the GPU
in tests/test_gpu_tuning.py)."""
import json

from paper_2606_30985_gb300 import autotune


def _table(tmp_path):
    table = {"version": 1, "classes": [
        {"chi_max": 16, "precision": "tf32x3", "gram_leg_splits": 32, "gram_rows_splits": 8},
        {"chi_max": 48, "precision": "tf32x3", "gram_leg_splits": 64, "gram_rows_splits": 16},
        {"chi_max": 100, "precision": "tf32x3", "gram_leg_splits": 128, "gram_rows_splits": 32},
        {"chi_max": 32, "precision": "fp32", "gram_leg_splits": 96, "gram_rows_splits": 64}]}
    p = tmp_path / "tuning.json"
    p.write_text(json.dumps(table))
    return str(p)


def test_lookup_picks_the_smallest_class_at_or_above_chi(tmp_path):
    p = _table(tmp_path)
    assert autotune.lookup(16, "tf32x3", p) == {"gram_leg_splits": 32, "gram_rows_splits": 8}
    assert autotune.lookup(17, "tf32x3", p) == {"gram_leg_splits": 64, "gram_rows_splits": 16}
    assert autotune.lookup(100, "tf32x3", p) == {"gram_leg_splits": 128, "gram_rows_splits": 32}
    # above every cached class: the largest
    assert autotune.lookup(128, "tf32x3", p) == {"gram_leg_splits": 128, "gram_rows_splits": 32}
    # precision classes are separate
    assert autotune.lookup(8, "fp32", p) == {"gram_leg_splits": 96, "gram_rows_splits": 64}
    assert autotune.lookup(8, "fp64", p) is None


def test_lookup_without_cache(tmp_path):
    assert autotune.lookup(16, "tf32x3", str(tmp_path / "missing.json")) is None
    bad = tmp_path / "bad.json"
    bad.write_text(json.dumps({"version": 2, "classes": []}))
    assert autotune.lookup(16, "tf32x3", str(bad)) is None
