"""The oracle against its stored regression fixtures (tests/golden/, written by
make_golden.py): a change of the oracle's arithmetic shows here first."""
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    a = np.loadtxt(os.path.join(HERE, name))
    return a[:, 0].astype(np.int64), a[:, 1:].T


def test_oracle_reproduces_config1_fixture():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    idx, ref = load("config1_xyz.txt")
    assert np.array_equal(idx, mg.IDX)
    got = mg.config1_xyz()
    np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())
