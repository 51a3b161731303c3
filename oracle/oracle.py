"""FP64 CPU oracle for the single-spin Metropolis sweep (ctypes front end).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this module; the product path
(the CUDA library and its Python binding) never does, and this module imports
nothing from the product package.

The arithmetic lives in ``hs_oracle.c`` (plain C, FP64, no FMA contraction);
this file only marshals numpy arrays.  What each function follows in the paper
(arXiv 2106.11286):

* ``energy``       -- Eq. 1, every nearest-neighbour bond once.
* ``sweep``        -- the Metropolis steps (i)-(iii), one colour class at a time.
* ``spin_sum`` / ``measure`` -- Eq. 2 (M = sum S_i / (N |S|), |S| = 1).
* ``philox``       -- Philox4x32-10 of Salmon et al. (SC'11), the counter-based
  generator both sides implement separately.

Every function here is pinned by the ``-m "not gpu"`` tests against closed
forms, invariants, brute force or an independent library routine.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODE_FP64 = 0   # two Philox calls, three 53-bit uniforms, FP64 spins
MODE_FP32 = 1   # one Philox block per two same-colour sites: 21/21/22-bit uniforms, FP64 spins
MODE_FP16 = 2   # FP32 schedule, trial spin rounded to binary16


def build(force: bool = False) -> str:
    """Compile ``hs_oracle.c`` into ``liboracle.so`` next to it (gcc)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i32p = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        dp = ctypes.POINTER(ctypes.c_double)
        L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.or_philox4x32_10.restype = None
        L.or_u53.argtypes = [ctypes.c_uint32, ctypes.c_uint32]
        L.or_u53.restype = ctypes.c_double
        L.or_u24.argtypes = [ctypes.c_uint32]
        L.or_u24.restype = ctypes.c_double
        L.or_round_half.argtypes = [ctypes.c_double]
        L.or_round_half.restype = ctypes.c_double
        for name in ("or_sc_neighbours", "or_bcc_neighbours", "or_fcc_neighbours"):
            f = getattr(L, name)
            f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, i32p]
            f.restype = ctypes.c_int64
        L.or_colour_structured.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p]
        L.or_colour_structured.restype = None
        L.or_colour_greedy.argtypes = [ctypes.c_int64, i64p, i32p, u8p, i32p]
        L.or_colour_greedy.restype = ctypes.c_int
        L.or_init_spins.argtypes = [ctypes.c_int64, u8p, ctypes.c_uint64, ctypes.c_uint32, dp]
        L.or_init_spins.restype = None
        L.or_sweep.argtypes = [ctypes.c_int64, i64p, i32p, i32p, ctypes.c_int, u8p,
                               ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_double,
                               ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                               ctypes.c_double, dp, dp, i64p, u8p]
        L.or_sweep.restype = ctypes.c_int64
        L.or_sweep_parallel.argtypes = L.or_sweep.argtypes + [ctypes.c_int]
        L.or_sweep_parallel.restype = ctypes.c_int64
        L.or_trial_uniforms.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                        ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, dp]
        L.or_trial_uniforms.restype = None
        L.or_sc_sites_neighbours.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int64, i64p, i64p]
        L.or_sc_sites_neighbours.restype = None
        L.or_init_sites.argtypes = [ctypes.c_int64, i64p, ctypes.c_uint64, ctypes.c_uint32, dp]
        L.or_init_sites.restype = None
        L.or_sc_sites_colour_rank.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int64, i64p, i32p,
                                              i64p]
        L.or_sc_sites_colour_rank.restype = None
        L.or_sites_update.argtypes = [ctypes.c_int64, i64p, i64p, i32p, dp, dp, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, dp, dp,
                                      ctypes.c_double, ctypes.c_double, u8p, u8p]
        L.or_sites_update.restype = None
        L.or_energy.argtypes = [ctypes.c_int64, i64p, i32p, u8p, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        L.or_energy.restype = ctypes.c_double
        L.or_spin_sum.argtypes = [ctypes.c_int64, u8p, dp, dp]
        L.or_spin_sum.restype = ctypes.c_int64
        _lib = L
    return _lib


def _p(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _tensor(A):
    """The on-site anisotropy tensor as the C side takes it: None, or the six
    entries (Axx, Ayy, Azz, Axy, Axz, Ayz) of the symmetric A in S^T A S
    (a 3x3 array is accepted and must be symmetric)."""
    if A is None:
        return None
    A = np.asarray(A, dtype=np.float64)
    if A.shape == (3, 3):
        assert np.array_equal(A, A.T)
        A = np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1], A[0, 2], A[1, 2]])
    assert A.shape == (6,)
    return np.ascontiguousarray(A)


# --------------------------------------------------------------------------- RNG
def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter under one 64-bit key (SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def u53(a: int, b: int) -> float:
    return lib().or_u53(a, b)


def u24(a: int) -> float:
    return lib().or_u24(a)


def round_half(x: float) -> float:
    return lib().or_round_half(x)


def trial_uniforms(mode: int, *, seed: int, replica: int, site: int, rank: int, sweep_index: int,
                   colour: int) -> tuple[float, float, float]:
    """(u_z, u_phi, P) of one trial move as the sweep draws them (Metropolis
    steps (ii)-(iii)): FP64 schedule keyed by the natural site index, FP32
    schedule by the site's rank in its colour class."""
    u = np.zeros(3, dtype=np.float64)
    lib().or_trial_uniforms(int(mode), int(seed), int(replica), int(site), int(rank), int(sweep_index), int(colour),
                            _p(u, ctypes.c_double))
    return float(u[0]), float(u[1]), float(u[2])


# --------------------------------------------------------------------------- lattices
class Graph:
    """Neighbour graph in natural site order (CSR), its colouring and mask."""

    def __init__(self, row_ptr, col, colour, n_colours, mask=None, z=None):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.colour = np.ascontiguousarray(colour, dtype=np.int32)
        self.n_colours = int(n_colours)
        self.mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        self.n = len(self.row_ptr) - 1
        self.z = z

    @property
    def n_present(self) -> int:
        return self.n if self.mask is None else int(self.mask.sum())


_KIND = {"sc": 0, "bcc": 1, "fcc": 2}
_BASIS = {"sc": 1, "bcc": 2, "fcc": 4}
_Z = {"sc": 6, "bcc": 8, "fcc": 12}


def neighbours(kind: str, dims, periodic: bool):
    """CSR neighbour list of an sc / bcc / fcc lattice in natural order."""
    Lx, Ly, Lz = (int(d) for d in dims)
    n = Lx * Ly * Lz * _BASIS[kind]
    f = getattr(lib(), f"or_{kind}_neighbours")
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    nnz = f(Lx, Ly, Lz, int(periodic), _p(row_ptr, ctypes.c_int64), None)
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    f(Lx, Ly, Lz, int(periodic), _p(row_ptr, ctypes.c_int64), _p(col, ctypes.c_int32))
    return row_ptr, col[:nnz]


def colour_structured(kind: str, dims) -> np.ndarray:
    Lx, Ly, Lz = (int(d) for d in dims)
    out = np.zeros(Lx * Ly * Lz * _BASIS[kind], dtype=np.int32)
    lib().or_colour_structured(_KIND[kind], Lx, Ly, Lz, _p(out, ctypes.c_int32))
    return out


def colour_greedy(row_ptr, col, mask=None):
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    n = len(row_ptr) - 1
    out = np.zeros(n, dtype=np.int32)
    nc = lib().or_colour_greedy(n, _p(row_ptr, ctypes.c_int64), _p(col, ctypes.c_int32),
                                _p(m, ctypes.c_uint8), _p(out, ctypes.c_int32))
    return out, nc


def lattice(kind: str, dims, periodic: bool = True, mask=None) -> Graph:
    """Structured lattice graph with its structural colouring."""
    row_ptr, col = neighbours(kind, dims, periodic)
    colour = colour_structured(kind, dims)
    nc = 2 if kind in ("sc", "bcc") else 4
    return Graph(row_ptr, col, colour, nc, mask, _Z[kind])


def csr_graph(row_ptr, col, mask=None) -> Graph:
    """User neighbour list with the greedy colouring."""
    colour, nc = colour_greedy(row_ptr, col, mask)
    return Graph(row_ptr, col, colour, nc, mask)


# --------------------------------------------------------------------------- method
def init_spins(g: Graph, seed: int, replica: int = 0) -> np.ndarray:
    S = np.zeros((g.n, 3), dtype=np.float64)
    lib().or_init_spins(g.n, _p(g.mask, ctypes.c_uint8), seed, replica, _p(S, ctypes.c_double))
    return S


def sweep(g: Graph, S: np.ndarray, *, J: float, K: float, e, beta: float, seed: int,
          sweep_index: int, replica: int = 0, mode: int = MODE_FP64, band: float = 0.0,
          band_site: np.ndarray | None = None, A=None):
    """One Metropolis sweep in place.  Returns (accepted, sum of accepted dH, band count).
    A: optional on-site anisotropy tensor (see _tensor)."""
    assert S.dtype == np.float64 and S.flags.c_contiguous and S.shape == (g.n, 3)
    ev = np.ascontiguousarray(e, dtype=np.float64)
    ev = ev / np.linalg.norm(ev)
    At = _tensor(A)
    sdh = ctypes.c_double(0.0)
    nb = ctypes.c_int64(0)
    acc = lib().or_sweep(g.n, _p(g.row_ptr, ctypes.c_int64), _p(g.col, ctypes.c_int32),
                         _p(g.colour, ctypes.c_int32), g.n_colours, _p(g.mask, ctypes.c_uint8),
                         float(J), float(K), _p(ev, ctypes.c_double), _p(At, ctypes.c_double), float(beta), int(seed),
                         int(replica), int(sweep_index), int(mode), float(band),
                         _p(S, ctypes.c_double), ctypes.byref(sdh), ctypes.byref(nb),
                         _p(band_site, ctypes.c_uint8))
    return int(acc), sdh.value, nb.value


def sweep_parallel(g: Graph, S: np.ndarray, *, J: float, K: float, e, beta: float, seed: int,
                   sweep_index: int, replica: int = 0, mode: int = MODE_FP64, band: float = 0.0,
                   band_site: np.ndarray | None = None, A=None, threads: int | None = None):
    """``sweep`` with each colour class's sites shared among OpenMP threads
    (default: every core).  Spins, accepted count and band flags equal
    ``sweep``'s bit for bit; the sum of accepted dH is added in another order."""
    assert S.dtype == np.float64 and S.flags.c_contiguous and S.shape == (g.n, 3)
    ev = np.ascontiguousarray(e, dtype=np.float64)
    ev = ev / np.linalg.norm(ev)
    At = _tensor(A)
    sdh = ctypes.c_double(0.0)
    nb = ctypes.c_int64(0)
    acc = lib().or_sweep_parallel(g.n, _p(g.row_ptr, ctypes.c_int64), _p(g.col, ctypes.c_int32),
                                  _p(g.colour, ctypes.c_int32), g.n_colours, _p(g.mask, ctypes.c_uint8),
                                  float(J), float(K), _p(ev, ctypes.c_double), _p(At, ctypes.c_double), float(beta),
                                  int(seed), int(replica), int(sweep_index), int(mode), float(band),
                                  _p(S, ctypes.c_double), ctypes.byref(sdh), ctypes.byref(nb),
                                  _p(band_site, ctypes.c_uint8), int(threads or os.cpu_count() or 1))
    if acc < 0:
        raise MemoryError("or_sweep_parallel: rank array allocation failed")
    return int(acc), sdh.value, nb.value


def sc_site_neighbours(dims, periodic: bool, sites) -> np.ndarray:
    """sc neighbours of the given natural indices, order -x, +x, -y, +y, -z, +z
    (m x 6 int64, -1 where an open boundary drops one)."""
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 6), dtype=np.int64)
    lib().or_sc_sites_neighbours(int(dims[0]), int(dims[1]), int(dims[2]), int(bool(periodic)), len(sites),
                                 _p(sites, ctypes.c_int64), _p(out, ctypes.c_int64))
    return out


def init_sites(sites, seed: int, replica: int = 0) -> np.ndarray:
    """Initial spins (as init_spins draws them) of sampled natural indices."""
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    S = np.zeros((len(sites), 3), dtype=np.float64)
    lib().or_init_sites(len(sites), _p(sites, ctypes.c_int64), int(seed), int(replica), _p(S, ctypes.c_double))
    return S


def sc_sites_colour_rank(dims, sites):
    """Colour and colour-class rank (ascending natural index) of sampled
    sites of a periodic sc lattice with even Lx, without a whole-lattice
    array."""
    assert int(dims[0]) % 2 == 0
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    colour = np.empty(len(sites), dtype=np.int32)
    rank = np.empty(len(sites), dtype=np.int64)
    lib().or_sc_sites_colour_rank(int(dims[0]), int(dims[1]), int(dims[2]), len(sites), _p(sites, ctypes.c_int64),
                                  _p(colour, ctypes.c_int32), _p(rank, ctypes.c_int64))
    return colour, rank


def sites_update(sites, ranks, colours, h, S, *, J: float, K: float, e, beta: float, seed: int,
                 sweep_index: int, replica: int = 0, mode: int = MODE_FP64, band: float = 0.0, A=None):
    """Metropolis steps (ii)-(iii) at sampled sites whose local fields h (m x 3,
    step (i)) are given, exactly as one sweep applies them.  S (m x 3) is
    updated in place; returns (accepted, in_band) as bool arrays."""
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    ranks = np.ascontiguousarray(ranks, dtype=np.int64)
    colours = np.ascontiguousarray(colours, dtype=np.int32)
    h = np.ascontiguousarray(h, dtype=np.float64)
    assert S.dtype == np.float64 and S.flags.c_contiguous and S.shape == (len(sites), 3)
    ev = np.ascontiguousarray(e, dtype=np.float64)
    ev = ev / np.linalg.norm(ev)
    acc = np.zeros(len(sites), dtype=np.uint8)
    band_flag = np.zeros(len(sites), dtype=np.uint8)
    At = _tensor(A)
    lib().or_sites_update(len(sites), _p(sites, ctypes.c_int64), _p(ranks, ctypes.c_int64),
                          _p(colours, ctypes.c_int32), _p(h, ctypes.c_double), _p(S, ctypes.c_double), int(mode),
                          int(seed), int(replica), int(sweep_index), float(J), float(K), _p(ev, ctypes.c_double),
                          _p(At, ctypes.c_double), float(beta), float(band), _p(acc, ctypes.c_uint8),
                          _p(band_flag, ctypes.c_uint8))
    return acc.astype(bool), band_flag.astype(bool)


def energy(g: Graph, S: np.ndarray, *, J: float, K: float, e, A=None) -> float:
    ev = np.ascontiguousarray(e, dtype=np.float64)
    ev = ev / np.linalg.norm(ev)
    S = np.ascontiguousarray(S, dtype=np.float64)
    At = _tensor(A)
    return lib().or_energy(g.n, _p(g.row_ptr, ctypes.c_int64), _p(g.col, ctypes.c_int32),
                           _p(g.mask, ctypes.c_uint8), float(J), float(K),
                           _p(ev, ctypes.c_double), _p(At, ctypes.c_double), _p(S, ctypes.c_double))


def spin_sum(g: Graph, S: np.ndarray):
    S = np.ascontiguousarray(S, dtype=np.float64)
    out = np.zeros(3, dtype=np.float64)
    n = lib().or_spin_sum(g.n, _p(g.mask, ctypes.c_uint8), _p(S, ctypes.c_double), _p(out, ctypes.c_double))
    return out, int(n)


def measure(g: Graph, S: np.ndarray, *, J: float, K: float, e, A=None) -> dict:
    """Instantaneous observables: E (Eq. 1) and M (Eq. 2, |S| = 1) with its moments."""
    E = energy(g, S, J=J, K=K, e=e, A=A)
    tot, n = spin_sum(g, S)
    M = tot / n
    absM = float(np.sqrt(M @ M))
    ev = np.asarray(e, dtype=np.float64)
    ev = ev / np.linalg.norm(ev)
    return {"E": E, "M": M, "absM": absM, "M2": absM ** 2, "M4": absM ** 4,
            "absMe": abs(float(M @ ev)), "n": n}
