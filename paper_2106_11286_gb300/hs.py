"""Thin ctypes binding of the C ABI in ``include/hs.h`` (same names, argument
marshalling only).  Every step of the Metropolis sweep runs in the CUDA
library ``libhs.so``; there is no Python or CPU fallback: if the library is
missing or fails to load, every call raises.

PyTorch is used only for plumbing: a ``torch.cuda.Stream`` (or its raw
handle) may be passed as the stream, and ``get_spins_device`` /
``set_spins_device`` accept CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

HS_SC, HS_BCC, HS_FCC, HS_CSR = 0, 1, 2, 3
HS_FP64, HS_FP32, HS_FP16 = 0, 1, 2
HS_INIT_RANDOM, HS_INIT_ALIGNED = 0, 1
HS_OK = 0
HS_N_MOMENTS = 9
STATUS = {0: "HS_OK", -1: "HS_E_INVALID", -2: "HS_E_CUDA", -3: "HS_E_OOM", -4: "HS_E_COLOUR",
          -5: "HS_E_TIMEOUT", -6: "HS_E_DEVICE"}
MOMENTS = ("sum_E", "sum_E2", "sum_absM", "sum_M2", "sum_M4", "sum_Mx", "sum_My", "sum_Mz", "sum_absMe")
TYPES = {"sc": HS_SC, "bcc": HS_BCC, "fcc": HS_FCC, "csr": HS_CSR}
PRECISIONS = {"fp64": HS_FP64, "fp32": HS_FP32, "fp16": HS_FP16}


class HSError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class hs_params(ctypes.Structure):
    _fields_ = [("J", ctypes.c_double), ("K", ctypes.c_double), ("e", ctypes.c_double * 3)]


class hs_measurement(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("M", ctypes.c_double * 3), ("absM", ctypes.c_double),
                ("M2", ctypes.c_double), ("M4", ctypes.c_double), ("n_sites", ctypes.c_int64),
                ("accept_rate", ctypes.c_double)]


class hs_launch(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("vec_width", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("tile_y", ctypes.c_int), ("prefetch", ctypes.c_int), ("order", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


HS_KERNEL_AUTO, HS_KERNEL_STENCIL, HS_KERNEL_TABLE, HS_KERNEL_MARCH, HS_KERNEL_PIPE = 0, 1, 3, 4, 5
KERNELS = {"auto": 0, "stencil": 1, "table": 3, "march": 4, "pipe": 5}


class hs_info(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("precision", ctypes.c_int), ("n_colours", ctypes.c_int),
                ("structured", ctypes.c_int), ("n_sites", ctypes.c_int64), ("n_present", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("sweep", ctypes.c_uint64), ("fold_sweeps", ctypes.c_int)]


_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); mirrors include/hs.h
SIGNATURES = {
    "hs_lattice_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i32p, ctypes.c_int, _i64p, _i32p,
                                         ctypes.c_int64, _u8p, ctypes.POINTER(hs_params), ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_uint32, _vp]),
    "hs_lattice_destroy": (None, [_vp]),
    "hs_init_spins": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hs_sweep": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int64]),
    "hs_sweep_pass": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int]),
    "hs_slab_create": (ctypes.c_int, [ctypes.POINTER(_vp), _i32p, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(hs_params), ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, _vp]),
    "hs_slab_plane": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp),
                                     ctypes.POINTER(ctypes.c_size_t)]),
    "hs_slab_copy_plane": (ctypes.c_int, [_vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int]),
    "hs_read_sums": (ctypes.c_int, [_vp, _dp]),
    "hs_get_sites": (ctypes.c_int, [_vp, ctypes.c_int64, _i64p, _dp]),
    "hs_measure": (ctypes.c_int, [_vp, ctypes.POINTER(hs_measurement)]),
    "hs_accumulate": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hs_reset_accumulator": (ctypes.c_int, [_vp]),
    "hs_read_accumulator": (ctypes.c_int, [_vp, _dp, _i64p]),
    "hs_get_spins": (ctypes.c_int, [_vp, _vp]),
    "hs_set_spins": (ctypes.c_int, [_vp, _vp]),
    "hs_get_spins_device": (ctypes.c_int, [_vp, _vp]),
    "hs_set_spins_device": (ctypes.c_int, [_vp, _vp]),
    "hs_set_spins_async": (ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    "hs_set_sweep_counter": (ctypes.c_int, [_vp, ctypes.c_uint64]),
    "hs_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(hs_info)]),
    "hs_enable_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hs_read_timing": (ctypes.c_int, [_vp, _dp, _i64p]),
    "hs_set_launch": (ctypes.c_int, [_vp, ctypes.POINTER(hs_launch)]),
    "hs_get_launch": (ctypes.c_int, [_vp, ctypes.POINTER(hs_launch)]),
    "hs_set_anisotropy_tensor": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "hs_get_anisotropy_tensor": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "hs_autotune": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int]),
    "hs_colour_greedy": (ctypes.c_int, [ctypes.c_int64, _i64p, _i32p, _u8p, _i32p, ctypes.POINTER(ctypes.c_int)]),
    "hs_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int]),
    "hs_batch_run": (ctypes.c_int, [_vp, _dp, ctypes.c_int64, ctypes.c_int64]),
    "hs_batch_destroy": (None, [_vp]),
    "hs_batch_autotune": (ctypes.c_int, [_vp, _dp, ctypes.c_int]),
    "hs_batch_get_layout": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "hs_batch_set_layout": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "hs_sweep_sc_fp32_noalloc": (ctypes.c_int, [_vp, _i32p, ctypes.POINTER(hs_params), ctypes.c_double,
                                                 ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                                 _vp, _vp]),
    "hs_batch_inject_timeout": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hs_measure_alu_peak": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_double)]),
    "hs_slab_pack": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp]),
    "hs_sweep_pass_part": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    "hs_slab_reserve_ctas": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "hs_slab_set_comm_stream": (ctypes.c_int, [_vp, _vp]),
    "hs_slab_unpack": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp]),
    "hs_read_sums_device": (ctypes.c_int, [_vp, _vp]),
    "hs_accumulate_sums": (ctypes.c_int, [_vp, _vp, ctypes.c_int64]),
    "hs_last_error": (ctypes.c_char_p, []),
    "hs_api_version": (ctypes.c_int, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhs.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run paper_2106_11286_gb300.build.build()")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code: int):
    if code != HS_OK:
        raise HSError(code, load().hs_last_error().decode())


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _ptr(a, ctype):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctype))


# ------------------------------------------------------------ functions (same names as the C ABI)
def hs_lattice_create(type, dims=None, periodic=True, row_ptr=None, col_idx=None, n_sites=0, site_mask=None,
                      J=1.0, K=0.0, e=(0.0, 0.0, 1.0), precision=HS_FP64, seed=0, replica=0, stream=None):
    L = load()
    t = TYPES[type] if isinstance(type, str) else int(type)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    d = None if dims is None else np.ascontiguousarray(dims, dtype=np.int32)
    rp = None if row_ptr is None else np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = None if col_idx is None else np.ascontiguousarray(col_idx, dtype=np.int32)
    if rp is not None:
        n_sites = len(rp) - 1
        if ci is None or len(ci) == 0:
            ci = np.zeros(1, dtype=np.int32)
    m = None if site_mask is None else np.ascontiguousarray(site_mask, dtype=np.uint8)
    p = hs_params(float(J), float(K), (ctypes.c_double * 3)(*[float(v) for v in e]))
    h = _vp()
    _check(L.hs_lattice_create(ctypes.byref(h), t, _ptr(d, ctypes.c_int32), int(bool(periodic)),
                               _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), int(n_sites),
                               _ptr(m, ctypes.c_uint8), ctypes.byref(p), prec, int(seed), int(replica),
                               _stream_handle(stream)))
    return h


def hs_lattice_destroy(h):
    load().hs_lattice_destroy(h)


def hs_init_spins(h, mode=HS_INIT_RANDOM):
    _check(load().hs_init_spins(h, int(mode)))


def hs_sweep(h, beta, n_sweeps=1):
    _check(load().hs_sweep(h, float(beta), int(n_sweeps)))


def hs_sweep_pass(h, beta, colour):
    _check(load().hs_sweep_pass(h, float(beta), int(colour)))


# parts of a slab's colour pass (hs_sweep_pass_part)
HS_PART_WHOLE, HS_PART_BOUNDARY, HS_PART_INTERIOR = 0, 1, 2


def hs_sweep_pass_part(h, beta, colour, part):
    _check(load().hs_sweep_pass_part(h, float(beta), int(colour), int(part)))


def hs_slab_reserve_ctas(h, ctas):
    _check(load().hs_slab_reserve_ctas(h, int(ctas)))


def hs_slab_set_comm_stream(h, stream):
    """Stream of the slab's pack / unpack / plane copies (a torch.cuda.Stream,
    a raw handle, or None for the legacy default stream)."""
    _check(load().hs_slab_set_comm_stream(h, _stream_handle(stream)))


def hs_slab_create(dims, z0, nz, J=1.0, K=0.0, e=(0.0, 0.0, 1.0), precision=HS_FP64, seed=0, replica=0,
                   stream=None):
    L = load()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    d = np.ascontiguousarray(dims, dtype=np.int32)
    p = hs_params(float(J), float(K), (ctypes.c_double * 3)(*[float(v) for v in e]))
    h = _vp()
    _check(L.hs_slab_create(ctypes.byref(h), _ptr(d, ctypes.c_int32), int(z0), int(nz), ctypes.byref(p), prec,
                            int(seed), int(replica), _stream_handle(stream)))
    return h


# slab plane selectors of hs_slab_plane / hs_slab_copy_plane
HALO_BELOW, FIRST_OWN, LAST_OWN, HALO_ABOVE = 0, 1, 2, 3


def hs_slab_plane(h, colour, component, which):
    ptr, nbytes = _vp(), ctypes.c_size_t(0)
    _check(load().hs_slab_plane(h, int(colour), int(component), int(which), ctypes.byref(ptr), ctypes.byref(nbytes)))
    return ptr.value, nbytes.value


def hs_slab_copy_plane(dst, dst_which, src, src_which, colour):
    _check(load().hs_slab_copy_plane(dst, int(dst_which), src, int(src_which), int(colour)))


def hs_slab_pack(h, colour, which, d_buf):
    """Copy the three component planes of one boundary / halo plane into the
    device buffer d_buf (a CUDA tensor or a device address)."""
    _check(load().hs_slab_pack(h, int(colour), int(which), _dev_ptr(d_buf)))


def hs_slab_unpack(h, colour, which, d_buf):
    _check(load().hs_slab_unpack(h, int(colour), int(which), _dev_ptr(d_buf)))


def hs_read_sums_device(h, d_out):
    _check(load().hs_read_sums_device(h, _dev_ptr(d_out)))


def hs_accumulate_sums(h, d_tot, n_sites):
    _check(load().hs_accumulate_sums(h, _dev_ptr(d_tot), int(n_sites)))


def _dev_ptr(x) -> int:
    return x.data_ptr() if hasattr(x, "data_ptr") else int(x)


def hs_get_sites(h, sites) -> np.ndarray:
    idx = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.zeros((len(idx), 3), dtype=np.float64)
    _check(load().hs_get_sites(h, len(idx), _ptr(idx, ctypes.c_int64), _ptr(out, ctypes.c_double)))
    return out


def hs_read_sums(h) -> np.ndarray:
    out = np.zeros(5, dtype=np.float64)
    _check(load().hs_read_sums(h, _ptr(out, ctypes.c_double)))
    return out


def hs_measure(h) -> dict:
    m = hs_measurement()
    _check(load().hs_measure(h, ctypes.byref(m)))
    return {"E": m.E, "M": np.array(list(m.M)), "absM": m.absM, "M2": m.M2, "M4": m.M4,
            "n_sites": m.n_sites, "accept_rate": m.accept_rate}


def hs_accumulate(h, on=True):
    _check(load().hs_accumulate(h, int(bool(on))))


def hs_reset_accumulator(h):
    _check(load().hs_reset_accumulator(h))


def hs_read_accumulator(h):
    buf = np.zeros(HS_N_MOMENTS, dtype=np.float64)
    cnt = ctypes.c_int64(0)
    _check(load().hs_read_accumulator(h, _ptr(buf, ctypes.c_double), ctypes.byref(cnt)))
    return buf, cnt.value


def hs_get_info(h) -> hs_info:
    info = hs_info()
    _check(load().hs_get_info(h, ctypes.byref(info)))
    return info


def hs_get_spins(h, out: np.ndarray | None = None) -> np.ndarray:
    info = hs_get_info(h)
    if out is None:
        out = np.empty((info.n_sites, 3), dtype=np.float64)
    assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == 3 * info.n_sites
    _check(load().hs_get_spins(h, out.ctypes.data))
    return out


def hs_set_spins(h, xyz: np.ndarray):
    info = hs_get_info(h)
    a = np.ascontiguousarray(xyz, dtype=np.float64)
    assert a.size == 3 * info.n_sites
    _check(load().hs_set_spins(h, a.ctypes.data))


def hs_get_spins_device(h, out):
    """out: contiguous float64 CUDA tensor with 3 * n_sites elements."""
    _check(load().hs_get_spins_device(h, out.data_ptr()))
    return out


def hs_set_spins_device(h, xyz):
    _check(load().hs_set_spins_device(h, xyz.data_ptr()))


def hs_set_spins_async(h, xyz):
    """xyz: contiguous host array (numpy, or a CPU torch tensor, ideally pinned)
    of 3 * n_sites float64 or float32 values in natural order.  Returns at once;
    the caller keeps xyz alive and unchanged until a later synchronous call on
    the handle has returned."""
    info = hs_get_info(h)
    if isinstance(xyz, np.ndarray):
        if not xyz.flags.c_contiguous:
            raise ValueError("xyz must be contiguous")
        dt, ptr, size = xyz.dtype, xyz.ctypes.data, xyz.size
        dtype = {np.dtype(np.float64): HS_FP64, np.dtype(np.float32): HS_FP32}.get(np.dtype(dt))
    else:
        if xyz.device.type != "cpu" or not xyz.is_contiguous():
            raise ValueError("xyz must be a contiguous host tensor")
        ptr, size = xyz.data_ptr(), xyz.numel()
        dtype = {"torch.float64": HS_FP64, "torch.float32": HS_FP32}.get(str(xyz.dtype))
    if dtype is None:
        raise ValueError("xyz must hold float64 or float32 values")
    if size != 3 * info.n_sites:
        raise ValueError(f"xyz holds {size} values, the lattice {3 * info.n_sites}")
    _check(load().hs_set_spins_async(h, ptr, dtype))


def hs_set_sweep_counter(h, sweep: int):
    _check(load().hs_set_sweep_counter(h, int(sweep)))


def hs_enable_timing(h, on=True):
    _check(load().hs_enable_timing(h, int(bool(on))))


def hs_read_timing(h):
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(load().hs_read_timing(h, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def hs_set_launch(h, kernel=0, vec_width=0, blocks_per_sm=0, tile_y=0, prefetch=0, order=0):
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    cfg = hs_launch(k, int(vec_width), int(blocks_per_sm), int(tile_y), int(prefetch), int(order))
    _check(load().hs_set_launch(h, ctypes.byref(cfg)))


def hs_get_launch(h) -> dict:
    cfg = hs_launch()
    _check(load().hs_get_launch(h, ctypes.byref(cfg)))
    return cfg.as_dict()


def tensor_entries(A):
    """The six entries (Axx, Ayy, Azz, Axy, Axz, Ayz) of a symmetric on-site
    anisotropy tensor given as six numbers or a symmetric 3x3 array."""
    A = np.asarray(A, dtype=np.float64)
    if A.shape == (3, 3):
        if not np.array_equal(A, A.T):
            raise ValueError("the anisotropy tensor must be symmetric")
        A = np.array([A[0, 0], A[1, 1], A[2, 2], A[0, 1], A[0, 2], A[1, 2]])
    if A.shape != (6,):
        raise ValueError("the anisotropy tensor takes 6 entries or a 3x3 array")
    return np.ascontiguousarray(A)


def hs_set_anisotropy_tensor(h, A):
    """-sum_i S_i^T A S_i on every site (A = None removes the term)."""
    if A is None:
        _check(load().hs_set_anisotropy_tensor(h, None))
        return
    t = tensor_entries(A)
    _check(load().hs_set_anisotropy_tensor(h, _ptr(t, ctypes.c_double)))


def hs_get_anisotropy_tensor(h) -> np.ndarray:
    t = np.zeros(6, dtype=np.float64)
    _check(load().hs_get_anisotropy_tensor(h, _ptr(t, ctypes.c_double)))
    return t


def hs_autotune(h, beta, n_trial_sweeps=3):
    _check(load().hs_autotune(h, float(beta), int(n_trial_sweeps)))


def hs_colour_greedy(row_ptr, col_idx, site_mask=None):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    if len(ci) == 0:
        ci = np.zeros(1, dtype=np.int32)
    m = None if site_mask is None else np.ascontiguousarray(site_mask, dtype=np.uint8)
    n = len(rp) - 1
    out = np.zeros(max(n, 1), dtype=np.int32)
    nc = ctypes.c_int(0)
    _check(load().hs_colour_greedy(n, _ptr(rp, ctypes.c_int64), _ptr(ci, ctypes.c_int32), _ptr(m, ctypes.c_uint8),
                                   _ptr(out, ctypes.c_int32), ctypes.byref(nc)))
    return out[:n], nc.value


def hs_sweep_sc_fp32_noalloc(planes, dims, beta, n_sweeps, d_out, *, J=1.0, K=0.0, e=(0.0, 0.0, 1.0), seed=0,
                             replica=0, first_sweep=0, stream=None):
    """planes: CUDA float32 tensor (6 * Lz * Ly * Lx/2, stencil layout); d_out:
    CUDA float64 tensor with HS_N_MOMENTS + 2 elements.  Allocates nothing.
    Both are checked (dtype, device, contiguity, size) before the call; the
    library checks the pointers' alignment."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    if d.shape != (3,):
        raise ValueError("dims must hold three sizes")
    want = 6 * int(d[2]) * int(d[1]) * (int(d[0]) // 2)
    for name, t, dtype, numel_ok in (("planes", planes, "torch.float32", lambda n: n == want),
                                     ("d_out", d_out, "torch.float64", lambda n: n >= HS_N_MOMENTS + 2)):
        if str(t.dtype) != dtype or t.device.type != "cuda" or not t.is_contiguous() or not numel_ok(t.numel()):
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of "
                             + (f"{want} elements" if name == "planes" else f"at least {HS_N_MOMENTS + 2} elements")
                             + f", got {t.dtype} on {t.device} with {t.numel()} elements")
    p = hs_params(float(J), float(K), (ctypes.c_double * 3)(*[float(v) for v in e]))
    _check(load().hs_sweep_sc_fp32_noalloc(planes.data_ptr(), _ptr(d, ctypes.c_int32), ctypes.byref(p),
                                           float(beta), int(seed), int(replica), int(first_sweep), int(n_sweeps),
                                           d_out.data_ptr(), _stream_handle(stream)))


ALU_FP64, ALU_FP32, ALU_FP32X2 = 0, 1, 2


def hs_measure_alu_peak(kind, stream=None) -> float:
    """Measured FLOP/s of DFMA (kind 0), FFMA (1) or packed FFMA2 (2) chains on
    every SM of the current device."""
    v = ctypes.c_double(0.0)
    _check(load().hs_measure_alu_peak(int(kind), _stream_handle(stream), ctypes.byref(v)))
    return v.value


def hs_batch_create(members):
    arr = (_vp * len(members))(*[m.value if isinstance(m, _vp) else m for m in members])
    b = _vp()
    _check(load().hs_batch_create(ctypes.byref(b), arr, len(members)))
    return b


def hs_batch_run(b, betas, n_sweeps, n_equil=0):
    bt = np.ascontiguousarray(betas, dtype=np.float64)
    _check(load().hs_batch_run(b, _ptr(bt, ctypes.c_double), int(n_sweeps), int(n_equil)))


def hs_batch_autotune(b, betas, n_trial_sweeps=3):
    bt = np.ascontiguousarray(betas, dtype=np.float64)
    _check(load().hs_batch_autotune(b, _ptr(bt, ctypes.c_double), int(n_trial_sweeps)))
    return hs_batch_get_layout(b)


def hs_batch_get_layout(b) -> dict:
    c = ctypes.c_int(0)
    a = ctypes.c_int(0)
    pf = ctypes.c_int(0)
    sc = ctypes.c_int(0)
    _check(load().hs_batch_get_layout(b, ctypes.byref(c), ctypes.byref(a), ctypes.byref(pf), ctypes.byref(sc)))
    return {"ctas_per_sm": c.value, "align_rows": a.value, "prefetch": pf.value, "schedule": sc.value}


def hs_batch_set_layout(b, ctas_per_sm, align_rows=0, prefetch=0, schedule=0):
    _check(load().hs_batch_set_layout(b, int(ctas_per_sm), int(align_rows), int(prefetch), int(schedule)))


def hs_batch_destroy(b):
    load().hs_batch_destroy(b)


def hs_batch_inject_timeout(b, on=True):
    _check(load().hs_batch_inject_timeout(b, int(bool(on))))


# ------------------------------------------------------------ convenience wrapper
class Lattice:
    """Owning wrapper: ``Lattice("sc", dims=(16,16,16), J=1, K=0.1, precision="fp64", seed=1)``."""

    def __init__(self, type, A=None, **kw):
        self.h = hs_lattice_create(type, **kw)
        if A is not None:
            try:
                hs_set_anisotropy_tensor(self.h, A)
            except Exception:
                self.close()
                raise

    def close(self):
        if self.h:
            hs_lattice_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def init(self, mode=HS_INIT_RANDOM):
        hs_init_spins(self.h, mode)

    def sweep(self, beta, n=1):
        hs_sweep(self.h, beta, n)

    def get_sites(self, sites):
        return hs_get_sites(self.h, sites)

    def measure(self):
        return hs_measure(self.h)

    def accumulate(self, on=True):
        hs_accumulate(self.h, on)

    def reset_accumulator(self):
        hs_reset_accumulator(self.h)

    def read_accumulator(self):
        return hs_read_accumulator(self.h)

    def get_spins(self):
        return hs_get_spins(self.h)

    def set_spins(self, xyz):
        hs_set_spins(self.h, xyz)

    def set_spins_async(self, xyz):
        hs_set_spins_async(self.h, xyz)

    def set_sweep_counter(self, s):
        hs_set_sweep_counter(self.h, s)

    def autotune(self, beta, n_trial_sweeps=3):
        hs_autotune(self.h, beta, n_trial_sweeps)
        return hs_get_launch(self.h)

    def set_launch(self, **cfg):
        hs_set_launch(self.h, **cfg)

    def set_anisotropy_tensor(self, A):
        hs_set_anisotropy_tensor(self.h, A)

    @property
    def launch(self):
        return hs_get_launch(self.h)

    @property
    def info(self):
        return hs_get_info(self.h)


class Slab(Lattice):
    """Owning wrapper of a z-slab: ``Slab(dims, z0, nz, J=.., precision=.., seed=..)``."""

    def __init__(self, dims, z0, nz, A=None, **kw):
        self.h = hs_slab_create(dims, z0, nz, **kw)
        if A is not None:
            try:
                hs_set_anisotropy_tensor(self.h, A)
            except Exception:
                self.close()
                raise

    def sweep_pass(self, beta, colour):
        hs_sweep_pass(self.h, beta, colour)

    def sweep_part(self, beta, colour, part):
        hs_sweep_pass_part(self.h, beta, colour, part)

    def reserve_ctas(self, ctas):
        hs_slab_reserve_ctas(self.h, ctas)

    def set_comm_stream(self, stream):
        hs_slab_set_comm_stream(self.h, stream)

    def read_sums(self):
        return hs_read_sums(self.h)
