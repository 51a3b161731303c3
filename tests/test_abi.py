"""CPU checks of the C-ABI library: it builds, loads and exports every entry
point that include/hs.h declares; host-only logic (greedy colouring, argument
validation) works without a GPU and agrees with the oracle's independent
implementation of the same colouring rule."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2106_11286_gb300 import hs, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hs_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hs_lattice_create", "hs_sweep", "hs_measure", "hs_lattice_destroy", "hs_get_spins",
                     "hs_set_spins", "hs_read_accumulator", "hs_batch_run", "hs_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = hs.load().__dict__.get("_name") or hs.library_path()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (hs_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    # and the Python binding binds exactly the declared set
    assert set(hs.SIGNATURES) == set(declared_functions())
    assert hs.load().hs_api_version() == 1


@pytest.mark.parametrize("graph", ["sphere", "chain", "sc_open", "fcc", "odd_ring"])
def test_greedy_colouring_matches_oracle(orc, graph):
    mask = None
    if graph == "sphere":
        rp, col, mask = inputs.bcc_nanoparticle(radius=5.0, box=12, vacancy_fraction=0.1, seed=4)
    elif graph == "chain":
        rp, col = inputs.open_chain(101)
    elif graph == "sc_open":
        rp, col = orc.neighbours("sc", (5, 7, 3), False)
    elif graph == "fcc":
        rp, col = orc.neighbours("fcc", (3, 3, 3), True)
    else:
        rp, col = orc.neighbours("sc", (5, 4, 4), True)
    got, nc = hs.hs_colour_greedy(rp, col, mask)
    want, nc_want = orc.colour_greedy(rp, col, mask)
    assert nc == nc_want
    assert np.array_equal(got, want)


def test_greedy_colouring_rejects_bad_lists():
    rp = np.array([0, 1, 2], dtype=np.int64)
    with pytest.raises(hs.HSError):
        hs.hs_colour_greedy(rp, np.array([0, 0], dtype=np.int32))   # self loop
    with pytest.raises(hs.HSError):
        hs.hs_colour_greedy(rp, np.array([1, 5], dtype=np.int32))   # out of range
    with pytest.raises(hs.HSError):
        hs.hs_colour_greedy(np.array([0, 2, 1], dtype=np.int64), np.array([1, 0], dtype=np.int32))


def test_create_validates_before_touching_the_device():
    # these fail in argument checking, with or without a GPU
    with pytest.raises(hs.HSError) as ei:
        hs.hs_lattice_create("sc", dims=(6, 5, 4))
    assert ei.value.code == -4           # HS_E_COLOUR: odd periodic sc
    with pytest.raises(hs.HSError) as ei:
        hs.hs_lattice_create("sc", dims=(4, 4, 4), e=(0, 0, 0))
    assert ei.value.code == -1
    with pytest.raises(hs.HSError) as ei:
        hs.hs_lattice_create("sc", dims=(4, 4, 4), precision=7)
    assert ei.value.code == -1
    with pytest.raises(hs.HSError) as ei:
        hs.hs_lattice_create("csr", row_ptr=np.array([0, 1], np.int64), col_idx=np.array([0], np.int32))
    assert ei.value.code == -1


def test_no_gpu_reports_device_error():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hs.HSError) as ei:
        hs.hs_lattice_create("sc", dims=(4, 4, 4))
    assert ei.value.code in (-2, -6)
