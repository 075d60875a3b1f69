"""The bounds-checked build (compiled with FE_CHECKED) against the normal build.

There every chunked kernel validates its plan record in shared memory before using any
index in it, and every fixup kernel its partial ranges and destinations (FE_ERR_BOUNDS
and a skipped chunk or entity on failure). Running the same assemblies through both
builds and finding clean status words and bit-identical values shows that no index
leaves its buffer on these meshes and that the checks change no arithmetic; a record
corrupted on purpose, in the checked build only, shows that the checks are live.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from helpers import fe_or_skip

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_checked_build_matches_normal_build(tmp_path):
    fe = fe_or_skip()
    from paper_1401_3301_gb300 import build_ext
    build_ext.build(checked=True)
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, FE_GB300_CHECKED="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), path], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    got = dict(np.load(path))
    assert "bounds-checked" in str(got.pop("version"))
    assert "bounds-checked" not in fe.fe_version()
    # a corrupted plan record is reported (FE_ERR_BOUNDS, chunk 1) by every chunked kernel
    bad = {k: tuple(got.pop(k)) for k in list(got) if k.startswith("corrupted:")}
    assert len(bad) == 29, sorted(bad)
    for name, st in bad.items():
        assert st == (9, 1), (name, st)

    import checked_cases
    ref = checked_cases.run(fe)
    assert set(got) == set(ref)
    for name, v in ref.items():
        if name.startswith("status:"):
            assert tuple(got[name]) == (0, -1), (name, got[name])
            assert tuple(v) == (0, -1), (name, v)
        else:
            assert got[name].dtype == v.dtype and got[name].shape == v.shape, name
            np.testing.assert_array_equal(got[name].view(np.uint8), v.view(np.uint8), err_msg=name)
