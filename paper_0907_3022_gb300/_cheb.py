"""ctypes binding of ``include/cheb.h`` (argument marshalling only).

Every function here calls the C ABI of ``libcheb.so`` with the same name; device arrays are
torch tensors whose ``data_ptr()`` is passed through.  All arithmetic happens in the CUDA
library: there is no CPU fallback, and loading fails loudly if the library cannot be built
or found.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcheb.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "cheb.h")

CHEB_OK = 0
CHEB_ERR_INVALID = -1
CHEB_ERR_ALIGN = -2
CHEB_ERR_CUDA = -3
CHEB_ERR_NOMEM = -4
CHEB_ERR_UNSUPPORTED = -5
CHEB_ERR_ORDER = -6
CHEB_ERR_DIVERGED = -7
CHEB_ERR_STATE = -8

CHEB_C128, CHEB_C64 = 0, 1
CHEB_LAT1D, CHEB_HONEYCOMB_ZZ, CHEB_HOLSTEIN = 0, 1, 2
(CHEB_OBS_NORM2, CHEB_OBS_ENERGY, CHEB_OBS_PROB_COLS, CHEB_OBS_HOL_DENSITY,
 CHEB_OBS_HOL_PHONON, CHEB_OBS_HOL_CHI) = range(6)


class cheb_ham_desc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("n", ctypes.c_int64),
        ("dx", ctypes.c_double),
        ("nblocks", ctypes.c_int32),
        ("W", ctypes.POINTER(ctypes.c_int32)),
        ("L", ctypes.POINTER(ctypes.c_int32)),
        ("hop", ctypes.c_double),
        ("onsite", ctypes.c_void_p),
        ("onsite_per_vec", ctypes.c_int32),
        ("hol_sites", ctypes.c_int32),
        ("hol_nph", ctypes.c_int32),
        ("hol_periodic", ctypes.c_int32),
        ("omega0", ctypes.c_double),
        ("g", ctypes.c_double),
        ("sell_sigma", ctypes.c_int32),
        ("hol_g", ctypes.c_void_p),
        ("hol_matrix_free", ctypes.c_int32),
    ]


class cheb_step_model(ctypes.Structure):
    _fields_ = [
        ("useful_site_orders", ctypes.c_double),
        ("computed_site_orders", ctypes.c_double),
        ("smem_bytes", ctypes.c_double),
        ("dram_bytes", ctypes.c_double),
        ("l2_bytes", ctypes.c_double),
        ("launches", ctypes.c_int64),
    ]


CHEB_PEAK_SMEM_LOAD_GBS, CHEB_PEAK_FP64_GFLOPS, CHEB_PEAK_FP32_GFLOPS = 0, 1, 2


class ChebError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


_lock = threading.Lock()
_lib = None

_c = ctypes
_vp, _dp, _ip, _i64p, _u8p = (_c.c_void_p, _c.POINTER(_c.c_double), _c.POINTER(_c.c_int),
                              _c.POINTER(_c.c_int64), _c.POINTER(_c.c_uint8))

_SIGS = {
    "cheb_last_error": ([], _c.c_char_p),
    "cheb_strerror": ([_c.c_int], _c.c_char_p),
    "cheb_rescale": ([_c.c_double, _c.c_double, _c.c_double, _dp, _dp], _c.c_int),
    "cheb_coeffs": ([_c.c_double, _c.c_double, _c.c_double, _c.c_double, _c.c_int, _dp, _dp, _ip],
                    _c.c_int),
    "cheb_plan_create": ([_c.POINTER(_vp), _c.POINTER(cheb_ham_desc), _dp, _dp, _c.c_double,
                          _c.c_int, _c.c_int, _vp], _c.c_int),
    "cheb_plan_destroy": ([_vp], None),
    "cheb_plan_set_tol": ([_vp, _c.c_double, _c.c_int], _c.c_int),
    "cheb_plan_set_onsite": ([_vp, _vp], _c.c_int),
    "cheb_plan_info": ([_vp, _i64p, _ip, _ip], _c.c_int),
    "cheb_plan_block": ([_vp, _c.c_int, _dp, _dp, _ip, _i64p, _ip, _ip], _c.c_int),
    "cheb_step": ([_vp, _vp, _c.c_double], _c.c_int),
    "cheb_evolve": ([_vp, _vp, _c.c_double, _c.c_int, _c.c_int, _vp], _c.c_int),
    "cheb_sync": ([_vp], _c.c_int),
    "cheb_evolve_host": ([_vp, _vp, _c.c_int64, _vp, _c.c_int64, _c.c_int64, _c.c_double, _c.c_int],
                         _c.c_int),
    "cheb_evolve_td": ([_vp, _vp, _c.c_double, _c.c_int, _vp, _c.c_int64, _c.c_int, _vp],
                       _c.c_int),
    "cheb_observables": ([_vp, _vp, _c.c_int, _c.c_double, _vp], _c.c_int),
    "cheb_adjoint_potential": ([_vp, _vp, _c.c_double, _c.c_int, _vp, _c.c_int64, _vp, _vp, _vp],
                               _c.c_int),
    "cheb_holstein_dim_phonon": ([_c.c_int, _c.c_int], _c.c_int64),
    "cheb_holstein_rank": ([_c.c_int, _c.c_int, _u8p, _c.c_int, _i64p], _c.c_int),
    "cheb_holstein_unrank": ([_c.c_int, _c.c_int, _c.c_int64, _u8p, _ip], _c.c_int),
    "cheb_holstein_phonon_neighbors": ([_c.c_int, _c.c_int, _c.c_int64, _c.c_int64, _i64p,
                                        _i64p], _c.c_int),
    "cheb_tb_tiles": ([_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.POINTER(_c.c_int32),
                       _c.c_int64, _i64p], _c.c_int),
    "cheb_tb_tiles_padded": ([_c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int, _c.c_int,
                              _c.POINTER(_c.c_int32), _c.c_int64, _i64p], _c.c_int),
    "cheb_plan_set_blocking_kernel": ([_vp, _c.c_int, _c.c_int, _c.c_int, _c.c_int], _c.c_int),
    "cheb_plan_blocking_kernel": ([_vp, _ip], _c.c_int),
    "cheb_plan_set_blocking_grid": ([_vp, _c.c_int], _c.c_int),
    "cheb_autotune": ([_vp], _c.c_int),
    "cheb_plan_launch": ([_vp, _ip, _ip, _ip, _ip], _c.c_int),
    "cheb_plan_set_blocking": ([_vp, _c.c_int, _c.c_int, _c.c_int], _c.c_int),
    "cheb_plan_set_cluster": ([_vp, _c.c_int], _c.c_int),
    "cheb_plan_cluster": ([_vp, _ip], _c.c_int),
    "cheb_plan_blocking": ([_vp, _ip, _ip, _ip], _c.c_int),
    "cheb_plan_export_csr": ([_vp, _i64p, _i64p, _dp, _i64p], _c.c_int),
    "cheb_plan_launches": ([_vp], _c.c_int64),
    "cheb_plan_set_timing": ([_vp, _c.c_int], _c.c_int),
    "cheb_plan_kernel_stats": ([_vp, _dp, _i64p, _dp, _c.c_int], _c.c_int),
    "cheb_plan_step_model": ([_vp, _c.POINTER(cheb_step_model)], _c.c_int),
    "cheb_plan_sell_stats": ([_vp, _ip, _i64p, _i64p], _c.c_int),
    "cheb_measure_peak": ([_c.c_int, _vp, _dp], _c.c_int),
    "cheb_region_norm_noalloc": ([_vp, _c.c_int, _c.c_int64, _c.c_int32, _c.c_int, _c.c_int64, _vp,
                                  _vp], _c.c_int),
}


def header_functions() -> list[str]:
    """Names of the functions include/cheb.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cheb_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load libcheb.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build

            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"CUDA library missing: {LIB_PATH}")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def check(status: int, where: str) -> int:
    if status != CHEB_OK:
        msg = lib().cheb_last_error().decode()
        raise ChebError(status, where, msg)
    return status


# ---- host functions ------------------------------------------------------------------------
def cheb_rescale(emin: float, emax: float, alpha: float):
    a, b = ctypes.c_double(), ctypes.c_double()
    check(lib().cheb_rescale(emin, emax, alpha, ctypes.byref(a), ctypes.byref(b)), "cheb_rescale")
    return a.value, b.value


def cheb_coeffs(a: float, b: float, dt: float, tol: float = 1e-14, max_order: int = 100000):
    """(complex multipliers C_0..C_M as a list of (re, im), M)."""
    import numpy as np

    re = np.zeros(max_order + 1)
    im = np.zeros(max_order + 1)
    M = ctypes.c_int()
    check(lib().cheb_coeffs(a, b, dt, tol, max_order, re.ctypes.data_as(_dp),
                            im.ctypes.data_as(_dp), ctypes.byref(M)), "cheb_coeffs")
    m = M.value
    return re[: m + 1] + 1j * im[: m + 1], m


def cheb_holstein_dim_phonon(L: int, nph: int) -> int:
    return int(lib().cheb_holstein_dim_phonon(L, nph))


def cheb_holstein_rank(L: int, nph: int, occ, e: int) -> int:
    import numpy as np

    o = np.ascontiguousarray(occ, dtype=np.uint8)
    idx = ctypes.c_int64()
    check(lib().cheb_holstein_rank(L, nph, o.ctypes.data_as(_u8p), e, ctypes.byref(idx)),
          "cheb_holstein_rank")
    return idx.value


def cheb_holstein_unrank(L: int, nph: int, idx: int):
    import numpy as np

    o = np.zeros(L, dtype=np.uint8)
    e = ctypes.c_int()
    check(lib().cheb_holstein_unrank(L, nph, idx, o.ctypes.data_as(_u8p), ctypes.byref(e)),
          "cheb_holstein_unrank")
    return e.value, o


def cheb_holstein_phonon_neighbors(L: int, nph: int, p0: int, count: int):
    """(up, dn): int64 [count, L] phonon ranks of n + 1_e and n - 1_e (-1: not admissible)
    for the phonon configurations of ranks p0 .. p0 + count - 1."""
    import numpy as np

    up = np.zeros((count, L), dtype=np.int64)
    dn = np.zeros((count, L), dtype=np.int64)
    check(lib().cheb_holstein_phonon_neighbors(L, nph, p0, count, up.ctypes.data_as(_i64p),
                                               dn.ctypes.data_as(_i64p)),
          "cheb_holstein_phonon_neighbors")
    return up, dn


def cheb_tb_tiles(W: int, L: int, orders_per_launch: int, region_sites: int):
    """int32 [ntiles, 8]: (R0, R1, C0, C1, r0, r1, c0, c1) of each temporal-blocking tile of a
    W x L ribbon (region, then interior; rows and columns half-open)."""
    import numpy as np

    n = ctypes.c_int64()
    check(lib().cheb_tb_tiles(W, L, orders_per_launch, region_sites, None, 0, ctypes.byref(n)),
          "cheb_tb_tiles")
    out = np.zeros((n.value, 8), dtype=np.int32)
    check(lib().cheb_tb_tiles(W, L, orders_per_launch, region_sites,
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value,
                              ctypes.byref(n)), "cheb_tb_tiles")
    return out


def cheb_tb_tiles_padded(W: int, L: int, orders_per_launch: int, region_positions: int, align: int,
                         boxes: bool = False):
    """As cheb_tb_tiles for the register-run kernel's padded regions: int32 [ntiles, 10], the 8
    columns of cheb_tb_tiles, then the row stride S and box height BH (per tile, or with
    boxes=True the ribbon's common ones)."""
    import numpy as np

    n = ctypes.c_int64()
    check(lib().cheb_tb_tiles_padded(W, L, orders_per_launch, region_positions, align, int(boxes),
                                     None, 0, ctypes.byref(n)), "cheb_tb_tiles_padded")
    out = np.zeros((n.value, 10), dtype=np.int32)
    check(lib().cheb_tb_tiles_padded(W, L, orders_per_launch, region_positions, align, int(boxes),
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), n.value,
                                     ctypes.byref(n)), "cheb_tb_tiles_padded")
    return out


CHEB_TB_SITES, CHEB_TB_RUNS, CHEB_TB_RUNS_TMA = 0, 1, 2


# ---- plans ---------------------------------------------------------------------------------
def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return t.data_ptr()


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


class Plan:
    """Owns a ``cheb_plan*``; methods are the C ABI calls on it (same names, minus prefix)."""

    def __init__(self, desc: cheb_ham_desc, emin, emax, alpha: float, prec: int, nvec: int,
                 stream=None, keep=()):
        n = max(1, desc.nblocks)
        lo = (ctypes.c_double * n)(*[float(x) for x in emin])
        hi = (ctypes.c_double * n)(*[float(x) for x in emax])
        h = ctypes.c_void_p()
        self._stream = stream
        check(lib().cheb_plan_create(ctypes.byref(h), ctypes.byref(desc), lo, hi, alpha, prec,
                                     nvec, _stream_handle(stream)), "cheb_plan_create")
        self.handle = h
        self.prec = prec
        self.nvec = nvec
        self.kind = desc.kind
        self._keep = keep
        sites = ctypes.c_int64()
        nb = ctypes.c_int()
        check(lib().cheb_plan_info(h, ctypes.byref(sites), None, ctypes.byref(nb)), "cheb_plan_info")
        self.sites = sites.value
        self.nblocks = nb.value

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().cheb_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls --------------------------------------------------------------------------
    def step(self, psi, dt: float):
        check(lib().cheb_step(self.handle, _ptr(psi), dt), "cheb_step")

    def evolve(self, psi, dt: float, nsteps: int, obs_every: int = 0, obs=None):
        check(lib().cheb_evolve(self.handle, _ptr(psi), dt, nsteps, obs_every, _ptr(obs)),
              "cheb_evolve")

    def evolve_host(self, host_in, host_out, njobs: int, dt: float, nsteps: int,
                    in_stride: int | None = None, out_stride: int | None = None):
        """njobs independent states from host memory (contiguous CPU tensors or numpy arrays;
        pinned memory for overlapped copies).  Strides in bytes: None = one state per job
        (consecutive states), 0 = the same state for every job."""
        vb = self.sites * self.nvec * (16 if self.prec == CHEB_C128 else 8)

        def hbuf(t):
            if hasattr(t, "data_ptr"):
                if t.is_cuda or not t.is_contiguous():
                    raise ValueError("contiguous host tensor expected")
                return t.data_ptr(), t.numel() * t.element_size()
            if not t.flags["C_CONTIGUOUS"]:
                raise ValueError("contiguous host array expected")
            return t.ctypes.data, t.nbytes

        pin, nin = hbuf(host_in)
        pout, nout = hbuf(host_out)
        si = vb if in_stride is None else in_stride
        so = vb if out_stride is None else out_stride
        for n, st in ((nin, si), (nout, so)):
            if njobs > 0 and n < (njobs - 1) * st + vb:
                raise ValueError("host buffer smaller than the states the jobs address")
        check(lib().cheb_evolve_host(self.handle, pin, si, pout, so, njobs, dt, nsteps),
              "cheb_evolve_host")

    def evolve_td(self, psi, dt: float, nsteps: int, onsite_seq, stride: int | None = None,
                  obs_every: int = 0, obs=None):
        """H(t) piecewise constant: step s uses the on-site energies onsite_seq[s] (device
        float64 tensor [nsteps, ...], rows 16-byte aligned)."""
        if stride is None:
            stride = onsite_seq[0].numel() if nsteps > 0 else 0
        check(lib().cheb_evolve_td(self.handle, _ptr(psi), dt, nsteps, _ptr(onsite_seq), stride,
                                   obs_every, _ptr(obs)), "cheb_evolve_td")

    def sync(self):
        check(lib().cheb_sync(self.handle), "cheb_sync")

    def observables(self, psi, kind: int, param: float, out):
        check(lib().cheb_observables(self.handle, _ptr(psi), kind, param, _ptr(out)),
              "cheb_observables")

    def adjoint_potential(self, psi0, dt: float, nsteps: int, lambda_n=None, region_col: int = 0,
                          grad=None, lambda0=None, P=None):
        check(lib().cheb_adjoint_potential(self.handle, _ptr(psi0), dt, nsteps, _ptr(lambda_n),
                                           region_col, _ptr(grad), _ptr(lambda0), _ptr(P)),
              "cheb_adjoint_potential")

    def set_tol(self, tol: float, max_order: int = 100000):
        check(lib().cheb_plan_set_tol(self.handle, tol, max_order), "cheb_plan_set_tol")

    def set_onsite(self, onsite):
        self._keep = self._keep + (onsite,)
        check(lib().cheb_plan_set_onsite(self.handle, _ptr(onsite)), "cheb_plan_set_onsite")

    def block(self, q: int):
        a, b = ctypes.c_double(), ctypes.c_double()
        M, W, L = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        off = ctypes.c_int64()
        check(lib().cheb_plan_block(self.handle, q, ctypes.byref(a), ctypes.byref(b),
                                    ctypes.byref(M), ctypes.byref(off), ctypes.byref(W),
                                    ctypes.byref(L)), "cheb_plan_block")
        return dict(a=a.value, b=b.value, M=M.value, offset=off.value, W=W.value, L=L.value)

    def autotune(self):
        check(lib().cheb_autotune(self.handle), "cheb_autotune")

    def launch_shape(self):
        """(threads per block, sites per thread, grid, vectors per thread)."""
        t, s, g, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().cheb_plan_launch(self.handle, ctypes.byref(t), ctypes.byref(s),
                                     ctypes.byref(g), ctypes.byref(v)), "cheb_plan_launch")
        return t.value, s.value, g.value, v.value

    def set_blocking(self, orders_per_launch: int, sites_per_thread: int = 4, threads: int = 256):
        check(lib().cheb_plan_set_blocking(self.handle, orders_per_launch, sites_per_thread,
                                           threads), "cheb_plan_set_blocking")

    def set_blocking_kernel(self, orders_per_launch: int, sites_per_thread: int, threads: int,
                            kernel: int):
        check(lib().cheb_plan_set_blocking_kernel(self.handle, orders_per_launch, sites_per_thread,
                                                  threads, kernel), "cheb_plan_set_blocking_kernel")

    def set_blocking_grid(self, ctas: int):
        """CTAs of each blocked launch (0: the kernel's default)."""
        check(lib().cheb_plan_set_blocking_grid(self.handle, ctas), "cheb_plan_set_blocking_grid")

    def blocking_kernel(self) -> int:
        """CHEB_TB_SITES, CHEB_TB_RUNS or CHEB_TB_RUNS_TMA (CHEB_TB_SITES when blocking is off)."""
        v = ctypes.c_int()
        check(lib().cheb_plan_blocking_kernel(self.handle, ctypes.byref(v)),
              "cheb_plan_blocking_kernel")
        return v.value

    def set_cluster(self, ctas: int = 8):
        """Whole steps on a cluster of `ctas` CTAs (8 or 16; 0 or False: off)."""
        check(lib().cheb_plan_set_cluster(self.handle, int(ctas)), "cheb_plan_set_cluster")

    def cluster(self) -> int:
        """CTAs of the cluster running whole steps (0: off)."""
        v = ctypes.c_int()
        check(lib().cheb_plan_cluster(self.handle, ctypes.byref(v)), "cheb_plan_cluster")
        return v.value

    def blocking(self):
        """(orders per launch, sites per thread); (0, 0) when off."""
        return self.blocking_shape()[:2]

    def blocking_shape(self):
        """(orders per launch, sites per thread, threads per CTA); zeros when off."""
        s, t, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().cheb_plan_blocking(self.handle, ctypes.byref(s), ctypes.byref(t),
                                       ctypes.byref(n)), "cheb_plan_blocking")
        return s.value, t.value, n.value

    def launches(self) -> int:
        return int(lib().cheb_plan_launches(self.handle))

    def set_timing(self, enable: bool):
        check(lib().cheb_plan_set_timing(self.handle, int(enable)), "cheb_plan_set_timing")

    def kernel_stats(self, reset: bool = False):
        """(total ms, launches, algorithmic bytes) of the timed recurrence launches."""
        ms, n, by = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        check(lib().cheb_plan_kernel_stats(self.handle, ctypes.byref(ms), ctypes.byref(n),
                                           ctypes.byref(by), int(reset)), "cheb_plan_kernel_stats")
        return ms.value, n.value, by.value

    def sell_stats(self) -> dict:
        """cheb_plan_sell_stats: sigma, stored entries (with padding), off-diagonal entries."""
        sg, st, nz = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().cheb_plan_sell_stats(self.handle, ctypes.byref(sg), ctypes.byref(st),
                                         ctypes.byref(nz)), "cheb_plan_sell_stats")
        return {"sigma": sg.value, "stored": st.value, "offdiag": nz.value}

    def step_model(self) -> dict:
        """cheb_plan_step_model as a dict (work of one step of the current schedule)."""
        m = cheb_step_model()
        check(lib().cheb_plan_step_model(self.handle, ctypes.byref(m)), "cheb_plan_step_model")
        return {name: getattr(m, name) for name, _ in cheb_step_model._fields_}

    def export_csr(self):
        import numpy as np

        nnz = ctypes.c_int64()
        check(lib().cheb_plan_export_csr(self.handle, None, None, None, ctypes.byref(nnz)),
              "cheb_plan_export_csr")
        rp = np.zeros(self.sites + 1, dtype=np.int64)
        col = np.zeros(nnz.value, dtype=np.int64)
        val = np.zeros(nnz.value, dtype=np.float64)
        check(lib().cheb_plan_export_csr(self.handle, rp.ctypes.data_as(_i64p),
                                         col.ctypes.data_as(_i64p), val.ctypes.data_as(_dp),
                                         ctypes.byref(nnz)), "cheb_plan_export_csr")
        return rp, col, val


def cheb_measure_peak(kind: int, stream=None) -> float:
    """Peak measured by the library's micro-kernels on the current device: CHEB_PEAK_SMEM_LOAD_GBS
    (GB/s), CHEB_PEAK_FP64_GFLOPS or CHEB_PEAK_FP32_GFLOPS (GFLOP/s)."""
    v = ctypes.c_double()
    check(lib().cheb_measure_peak(int(kind), _stream_handle(stream), ctypes.byref(v)),
          "cheb_measure_peak")
    return v.value


def cheb_region_norm_noalloc(psi, prec: int, n_sites: int, L: int, nvec: int, col_min: int, out,
                             stream=None):
    """Plan-free region norm into out (device doubles [nvec]); allocates nothing."""
    check(lib().cheb_region_norm_noalloc(_ptr(psi), prec, n_sites, L, nvec, col_min, _ptr(out),
                                         _stream_handle(stream)), "cheb_region_norm_noalloc")


# ---- descriptor helpers ----------------------------------------------------------------------
def desc_lat1d(n: int, dx: float, onsite=None) -> cheb_ham_desc:
    d = cheb_ham_desc()
    d.kind = CHEB_LAT1D
    d.n = n
    d.dx = dx
    d.nblocks = 1
    d.onsite = _ptr(onsite)
    return d


def desc_ribbons(W, L, hop: float = 1.0, onsite=None, onsite_per_vec: bool = False):
    """Descriptor for len(W) zigzag ribbons; returns (desc, keep-alive arrays)."""
    n = len(W)
    Wa = (ctypes.c_int32 * n)(*[int(x) for x in W])
    La = (ctypes.c_int32 * n)(*[int(x) for x in L])
    d = cheb_ham_desc()
    d.kind = CHEB_HONEYCOMB_ZZ
    d.nblocks = n
    d.W = ctypes.cast(Wa, ctypes.POINTER(ctypes.c_int32))
    d.L = ctypes.cast(La, ctypes.POINTER(ctypes.c_int32))
    d.hop = hop
    d.onsite = _ptr(onsite)
    d.onsite_per_vec = int(onsite_per_vec)
    return d, (Wa, La, onsite)


def desc_armchair(n_a, lengths, hop: float, onsite=None, onsite_per_vec: bool = False):
    """Armchair ribbons (armchair edges along the length; n_a dimer lines across): the
    brick-wall operator of CHEB_HONEYCOMB_ZZ with the long direction across the rows,
    W = length, L = n_a.  Returns (descriptor, arrays to keep alive)."""
    return desc_ribbons(list(lengths), list(n_a), hop, onsite, onsite_per_vec)


def desc_holstein(L: int, nph: int, periodic: bool, hop: float, omega0: float, g: float,
                  delta=None, gsite=None, matrix_free: bool = False,
                  sell_sigma: int = 0) -> cheb_ham_desc:
    """Holstein descriptor; delta / gsite: optional device float64 tensors [L] with the site
    potentials Delta_i and couplings g_i (keep them alive while the plan is built);
    matrix_free: apply H without storing it (L <= 32, nph <= 15); sell_sigma: SELL-C-sigma
    sorting window of the stored matrix (0: library default, 1: none)."""
    d = cheb_ham_desc()
    d.kind = CHEB_HOLSTEIN
    d.nblocks = 1
    d.hop = hop
    d.hol_sites = L
    d.hol_nph = nph
    d.hol_periodic = int(periodic)
    d.omega0 = omega0
    d.g = g
    d.onsite = _ptr(delta)
    d.hol_g = _ptr(gsite)
    d.hol_matrix_free = int(matrix_free)
    d.sell_sigma = int(sell_sigma)
    return d
