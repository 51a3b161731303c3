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


def _words(orc, *, index, sweep_index, colour, call, replica, seed):
    """One Philox block of the trial schedule: counter (index, sweep,
    tag 0 << 24 | colour << 8 | call, replica), key (seed lo, seed hi)."""
    ctr = [index & 0xFFFFFFFF, sweep_index & 0xFFFFFFFF, (colour << 8) | call, replica]
    return [int(w) for w in orc.philox(ctr, [seed & 0xFFFFFFFF, seed >> 32])]


_DRAWS = [(seed, replica, rank, sweep_index, colour)
          for seed in (1, 2, 0x1234567890AB) for replica in (0, 5) for rank in (0, 1, 2, 3, 4097, 2 ** 31 + 1)
          for sweep_index in (0, 499) for colour in (0, 1, 3)]


def test_fp32_schedule_fields_exact(orc):
    """FP32/FP16 schedule: a site of class rank r takes half r & 1 of block
    r >> 1, words a = w[2(r&1)], b = w[2(r&1)+1]; u_z = (a >> 11) 2^-21,
    u_phi = (b >> 11) 2^-21, P = ((a & 0x7FF) << 11 | (b & 0x7FF)) 2^-22.
    Checked the other way round: the three uniforms, scaled to integers,
    must rebuild both words of the right half exactly, so a swapped half, a
    field taken twice from one word or a dropped bit fails."""
    for seed, replica, rank, sweep_index, colour in _DRAWS:
        uz, uphi, P = orc.trial_uniforms(1, seed=seed, replica=replica, site=12345, rank=rank,
                                         sweep_index=sweep_index, colour=colour)
        kz, kphi, kp = Fraction(uz) * 2 ** 21, Fraction(uphi) * 2 ** 21, Fraction(P) * 2 ** 22
        for k, top in ((kz, 2 ** 21), (kphi, 2 ** 21), (kp, 2 ** 22)):
            assert k.denominator == 1 and 0 <= k < top
        kz, kphi, kp = int(kz), int(kphi), int(kp)
        w = _words(orc, index=rank >> 1, sweep_index=sweep_index, colour=colour, call=0, replica=replica, seed=seed)
        half = rank & 1
        assert (kz << 11) | (kp >> 11) == w[2 * half]
        assert (kphi << 11) | (kp & 0x7FF) == w[2 * half + 1]
        # the site's natural index plays no part in this schedule
        assert orc.trial_uniforms(1, seed=seed, replica=replica, site=7, rank=rank, sweep_index=sweep_index,
                                  colour=colour) == (uz, uphi, P)
        # FP16 draws the same numbers
        assert orc.trial_uniforms(2, seed=seed, replica=replica, site=7, rank=rank, sweep_index=sweep_index,
                                  colour=colour) == (uz, uphi, P)


def test_fp32_schedule_halves_of_one_block_share_nothing(orc):
    """Ranks 2k and 2k+1 read disjoint halves of one block: together their six
    fields hold all 128 bits of it."""
    for k in (0, 1, 77):
        a = orc.trial_uniforms(1, seed=2, replica=0, site=0, rank=2 * k, sweep_index=3, colour=1)
        b = orc.trial_uniforms(1, seed=2, replica=0, site=0, rank=2 * k + 1, sweep_index=3, colour=1)
        w = _words(orc, index=k, sweep_index=3, colour=1, call=0, replica=0, seed=2)
        bits = []
        for uz, uphi, P in (a, b):
            kz, kphi, kp = int(uz * 2 ** 21), int(uphi * 2 ** 21), int(P * 2 ** 22)
            bits += [(kz << 11) | (kp >> 11), (kphi << 11) | (kp & 0x7FF)]
        assert bits == w


def test_fp64_schedule_fields_exact(orc):
    """FP64 schedule: keyed by the natural index; u_z from words 0, 1 and u_phi
    from words 2, 3 of call 0, P from words 0, 1 of call 1, each the 53-bit
    map (w0 >> 5) 2^26 + (w1 >> 6) over 2^53.  The uniforms, scaled to
    integers, must rebuild the top 27 + 26 bits of those words."""
    for seed, replica, site, sweep_index, colour in _DRAWS:
        uz, uphi, P = orc.trial_uniforms(0, seed=seed, replica=replica, site=site, rank=999,
                                         sweep_index=sweep_index, colour=colour)
        w0 = _words(orc, index=site, sweep_index=sweep_index, colour=colour, call=0, replica=replica, seed=seed)
        w1 = _words(orc, index=site, sweep_index=sweep_index, colour=colour, call=1, replica=replica, seed=seed)
        for u, (a, b) in ((uz, (w0[0], w0[1])), (uphi, (w0[2], w0[3])), (P, (w1[0], w1[1]))):
            k = Fraction(u) * 2 ** 53
            assert k.denominator == 1
            k = int(k)
            assert k >> 26 == a >> 5 and k & (2 ** 26 - 1) == b >> 6
