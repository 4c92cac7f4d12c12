"""The ctypes mirrors of the C-ABI structs match include/pepo.h byte for byte,
and the host-only trap check pepo_c_drop follows its stated rule.

The layout probe is a small C program compiled with the host compiler against
the header; it prints sizeof and every field's offset, which must equal what
ctypes computes for the binding's mirror structs (a mismatch would let the
library write past the arrays the binding allocates).
"""
import ctypes
import math
import os
import shutil
import subprocess

import pytest

import paper_2606_30985_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MIRRORS = {"pepo_config": pkg._Config, "pepo_diag": pkg._Diag, "pepo_tuning": pkg._Tuning}


def _probe_source():
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pepo.h"', "int main(void) {"]
    for cname, mirror in MIRRORS.items():
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for field, _ in mirror._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, field, cname, field))
    lines += ["  return 0;", "}"]
    return "\n".join(lines) + "\n"


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("layout")
    src, exe = d / "probe.c", d / "probe"
    src.write_text(_probe_source())
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for line in out.splitlines():
        name, field, value = line.split()
        table[(name, field)] = int(value)
    return table


@pytest.mark.parametrize("cname", sorted(MIRRORS))
def test_mirror_struct_matches_the_header(c_layout, cname):
    mirror = MIRRORS[cname]
    assert ctypes.sizeof(mirror) == c_layout[(cname, "sizeof")]
    for field, _ in mirror._fields_:
        assert getattr(mirror, field).offset == c_layout[(cname, field)], field


def test_c_drop_rule():
    lib = pkg.load_library()
    f = lib.pepo_c_drop
    assert f(0.20, 1e-6, 0.09, 1e-6) == 1          # more than halved, discarded weight flat
    assert f(0.20, 1e-6, 0.11, 1e-6) == 0          # dropped by less than half
    assert f(0.20, 1e-6, 0.09, 3e-6) == 0          # the discarded weight jumped (x3)
    assert f(0.20, 1e-6, 0.09, 1.9e-6) == 1        # grew, but by less than 2x
    assert f(-0.20, 0.0, 0.05, 0.0) == 1           # magnitudes; sign changes count
    assert f(0.20, 0.0, 0.05, 1e-13) == 1          # below the 1e-12 floor: no jump
    assert f(0.20, 0.0, 0.05, 1e-9) == 0
    assert f(0.05, 1e-6, 0.20, 1e-6) == 0          # a rise is no drop
    assert f(math.nan, 0.0, 0.01, 0.0) == 0 and f(0.2, 0.0, math.inf, 0.0) == 0
