"""The FP64 oracle reproduces its stored run of the homogeneous 8^3 cube
(``tests/golden/cube8_ngll5_seismograms.txt``, written by ``tests/golden/make_golden.py``
from the oracle alone): an anchor that makes any later change of the oracle's arithmetic
visible. The stored time step also equals its closed form, 0.4 * 62.5 m (1 - sqrt(3/7)) /
3000 m/s (the smallest GLL spacing of a 125 m element at NGLL 5 over vp, Courant 0.4)."""
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.slow
def test_oracle_reproduces_stored_cube_run():
    g = _golden()
    stored = g.read_cube8()
    _, ref = g.cube8()
    assert abs(stored["dt"] / (0.4 * 62.5 * (1.0 - np.sqrt(3.0 / 7.0)) / 3000.0) - 1.0) < 1e-13
    assert abs(ref["dt"] / stored["dt"] - 1.0) < 1e-14
    assert list(ref["src"]) == list(stored["src"]) and list(ref["rec"]) == list(stored["rec"])
    assert stored["seis"].shape == (8, 3, 200)
    scale = np.abs(stored["seis"]).max()
    assert np.abs(ref["seis"] - stored["seis"]).max() <= 1e-10 * scale
