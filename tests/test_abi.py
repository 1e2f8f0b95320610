"""The C-ABI library builds, loads and exports every symbol include/*.h
declares; parameter validation and footprints need no GPU."""
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(bfibm_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    bfibm.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", bfibm.library_path()],
                         capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = declared() - exported
    assert not missing, missing
    assert len(declared()) >= 30


def test_binding_covers_every_symbol():
    assert declared() == set(bfibm.SIGNATURES)


def test_footprint_and_validation_without_gpu():
    prm = W.c3()["params"]
    fp = bfibm.footprint(dict(prm, precision=0), 20000, 150000)
    cells = 128 * 128 * 256
    assert 25 * 8 * cells < fp < 60 * 8 * cells
    bad = dict(W.c1()["params"], phi_kind=3)
    with pytest.raises(bfibm.BfibmError) as e:
        bfibm.footprint(bad)
    assert e.value.status == bfibm.EINVAL
    for key, val in (("dim", 4), ("n", [63, 32, 1]), ("dt", 0.0), ("flow_axis", 1),
                     ("mu_ratio", 0.5)):
        with pytest.raises(bfibm.BfibmError):
            bfibm.footprint(dict(W.c1()["params"], **{key: val}))


def test_grids_beyond_32_bit_offsets_are_refused():
    # the kernels index within a level array with 32-bit offsets: a 3D grid
    # whose level-0 arrays would hold 2^31 elements or more is refused before
    # any allocation; the 1024^3 grid (about 1.08e9 elements) is not
    prm = W.c3()["params"]
    big = dict(prm, n=[2048, 1024, 1024])
    with pytest.raises(bfibm.BfibmError) as e:
        bfibm.footprint(big)
    assert e.value.status == bfibm.EINVAL
    assert bfibm.footprint(dict(prm, n=[1024, 1024, 1024]), 0, 0) > 0


def test_output_buffers_are_checked_before_the_library_writes():
    out = bfibm._out(None, (3, 4))
    assert out.shape == (3, 4) and out.dtype == np.float64
    good = np.zeros((3, 4))
    assert bfibm._out(good, (3, 4)) is good
    for bad in (np.zeros((4, 3)), np.zeros((3, 4), np.float32), np.zeros((4, 3)).T,
                np.zeros(12), [[0.0] * 4] * 3):
        with pytest.raises(ValueError):
            bfibm._out(bad, (3, 4))
    ro = np.zeros((3, 4))
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        bfibm._out(ro, (3, 4))
