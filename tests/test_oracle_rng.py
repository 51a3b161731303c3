"""Pins of the oracle's random-number layer.

* Philox4x32-10 against the published Random123 known-answer vectors and, on a
  random grid of counters and keys, against PyTorch's independent header-only
  ``at::philox_engine`` (compiled here with g++).
* The integer -> uniform conversions are exact and land in [0, 1).
* The binary16 rounding helper agrees with numpy's float16 conversion.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(orc):
    rows = _kat_rows()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = orc.philox(ctr, key)
        assert [int(x) for x in got] == want


@pytest.fixture(scope="module")
def torch_philox(tmp_path_factory):
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if shutil.which("g++") is None or not os.path.exists(
            os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("g++ or the torch headers are missing")
    exe = str(tmp_path_factory.mktemp("philox") / "philox_torch_ref")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", inc, os.path.join(HERE, "philox_torch_ref.cpp"),
                    "-o", exe], check=True)

    def run(rows):
        text = "".join(" ".join(f"{x:08x}" for x in r) + "\n" for r in rows)
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
        return [[int(t, 16) for t in line.split()] for line in out.strip().splitlines()]
    return run


def test_philox_matches_torch_engine(orc, torch_philox):
    rng = np.random.default_rng(12345)
    rows = rng.integers(0, 2 ** 32, size=(300, 6), dtype=np.uint64).tolist()
    # include the counter layouts the method uses: small site / sweep numbers
    for site in (0, 1, 4095, 16777215):
        for sweep in (0, 1, 499):
            for tag in (0, 1):
                for colour in (0, 1, 3):
                    for call in (0, 1):
                        rows.append([site, sweep, (tag << 24) | (colour << 8) | call, 7, 2, 0])
    want = torch_philox(rows)
    for r, w in zip(rows, want):
        got = orc.philox(r[0:4], r[4:6])
        assert [int(x) for x in got] == w, r


def test_uniform_conversions_exact(orc):
    assert orc.u53(0, 0) == 0.0
    assert orc.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert orc.u24(0) == 0.0
    assert orc.u24(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    rng = np.random.default_rng(7)
    for a, b in rng.integers(0, 2 ** 32, size=(2000, 2), dtype=np.uint64).tolist():
        u = orc.u53(a, b)
        assert Fraction(u) == Fraction((a >> 5) * 2 ** 26 + (b >> 6), 2 ** 53)
        assert 0.0 <= u < 1.0
        v = orc.u24(a)
        assert Fraction(v) == Fraction(a >> 8, 2 ** 24)
        assert 0.0 <= v < 1.0


def test_round_half_matches_numpy(orc):
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.uniform(-1, 1, 20000), rng.uniform(-1e-4, 1e-4, 2000),
                         [0.0, 1.0, -1.0, 0.99999, 2.0 ** -24, 3 * 2.0 ** -25, 65504.0]])
    # ties: exact midpoints between neighbouring halves must round to even
    h = np.float16(0.5) + np.arange(50, dtype=np.float16) * np.float16(2.0 ** -11)
    mids = (h[:-1].astype(np.float64) + h[1:].astype(np.float64)) / 2
    xs = np.concatenate([xs, mids, -mids])
    for x in xs:
        assert orc.round_half(float(x)) == float(np.float16(x)), x
