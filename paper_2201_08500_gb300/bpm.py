"""Thin ctypes binding of libbpm (include/bpm.h): argument marshalling only.

Every step of the BPM runs in the CUDA library; this module converts numpy
arrays / torch tensors to pointers and status codes to exceptions.  There is
no fallback: if libbpm.so cannot be loaded, or the device is not a GB300
(sm_103a), the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbpm.so")

BPM_FIELD_E0, BPM_FIELD_EH, BPM_FIELD_EH_TIME = 0, 1, 2
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "CUDA", 4: "UNSUPPORTED", 5: "TIMEOUT",
          6: "STATE", 7: "CANCELLED"}

# Every symbol include/bpm.h declares (checked by the CPU test suite).
EXPORTS = ("bpm_plan_create", "bpm_set_crystal", "bpm_set_pulse", "bpm_set_fields", "bpm_run",
           "bpm_sync", "bpm_fetch_fields", "bpm_fetch_reflectivity", "bpm_set_timing",
           "bpm_get_stats", "bpm_last_error", "bpm_plan_destroy", "bpm_version", "bpm_plan_bytes",
           "bpm_batch_create", "bpm_batch_submit", "bpm_batch_step", "bpm_batch_run",
           "bpm_batch_run_graph", "bpm_batch_poll", "bpm_batch_cancel", "bpm_batch_sync",
           "bpm_batch_info", "bpm_batch_last_error", "bpm_batch_destroy", "bpm_run_noalloc",
           "bpm_noalloc_scratch_bytes", "bpm_noalloc_last_error", "bpm_set_stream",
           "bpm_set_geometry", "bpm_batch_set_max_blocks", "bpm_batch_pending",
           "bpm_batch_graph_kernels", "bpm_get_launch", "bpm_set_launch", "bpm_tune",
           "bpm_tune_save", "bpm_tune_load", "bpm_tune_clear", "bpm_set_channel_shard",
           "bpm_set_crystal_shape", "bpm_measure_peak", "bpm_check_bounded_wait")


class BpmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("split_order", ctypes.c_int32),
                ("zassenhaus", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("march_ms", ctypes.c_double), ("launches", ctypes.c_int32),
                ("march_launches", ctypes.c_int32), ("threads_per_channel", ctypes.c_int32),
                ("channels_per_block", ctypes.c_int32), ("blocks", ctypes.c_int32),
                ("smem_bytes", ctypes.c_int32)]


class Launch(ctypes.Structure):
    """Launch form of a plan (see bpm_launch in include/bpm.h)."""
    _fields_ = [("form", ctypes.c_int32), ("channels_per_block", ctypes.c_int32),
                ("row_threads", ctypes.c_int32), ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class CrystalParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("chi0_re", "chi0_im", "chih_re", "chih_im",
                                               "chihbar_re", "chihbar_im", "theta_B", "lambda_B",
                                               "x_surface", "thickness")]


class BeamParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("theta_i", "x0", "w0", "zx", "zR")]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int


def load(path: str = LIB_PATH):
    """Load libbpm.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} is missing; build the CUDA library first "
                                "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(path)
    sig = {
        "bpm_plan_create": ([ctypes.POINTER(Grid), _I, _P, ctypes.POINTER(_P)], _I),
        "bpm_set_crystal": ([_P] + [_D] * 10 + [_P, _I], _I),
        "bpm_set_pulse": ([_P, _P, _P, _D, _D, _D, _D, _D], _I),
        "bpm_set_fields": ([_P, _P, _P, _I, _I], _I),
        "bpm_set_channel_shard": ([_P, _I, _I, _D], _I),
        "bpm_set_crystal_shape": ([_P, _P, _I], _I),
        "bpm_run": ([_P, _I], _I),
        "bpm_sync": ([_P], _I),
        "bpm_set_stream": ([_P, _P], _I),
        "bpm_set_geometry": ([_P, _D, _D, _D], _I),
        "bpm_batch_set_max_blocks": ([_P, _I], _I),
        "bpm_batch_pending": ([_P, ctypes.POINTER(ctypes.c_int)], _I),
        "bpm_batch_graph_kernels": ([_P, ctypes.POINTER(ctypes.c_int)], _I),
        "bpm_get_launch": ([_P, ctypes.POINTER(Launch)], _I),
        "bpm_set_launch": ([_P, ctypes.POINTER(Launch)], _I),
        "bpm_tune": ([ctypes.POINTER(Grid), _I, _I, ctypes.POINTER(Launch), ctypes.POINTER(Launch),
                      _I, ctypes.POINTER(_I)], _I),
        "bpm_tune_save": ([ctypes.c_char_p], _I),
        "bpm_tune_load": ([ctypes.c_char_p, ctypes.POINTER(_I)], _I),
        "bpm_tune_clear": ([], None),
        "bpm_fetch_fields": ([_P, _I, _P, ctypes.c_size_t, _I], _I),
        "bpm_fetch_reflectivity": ([_P, _P, _P, _P], _I),
        "bpm_set_timing": ([_P, _I], _I),
        "bpm_get_stats": ([_P, ctypes.POINTER(Stats)], _I),
        "bpm_last_error": ([_P], ctypes.c_char_p),
        "bpm_plan_destroy": ([_P], None),
        "bpm_version": ([], ctypes.c_char_p),
        "bpm_plan_bytes": ([ctypes.POINTER(Grid), _I, _I], ctypes.c_size_t),
        "bpm_measure_peak": ([_I, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_float), _P],
                             _I),
        "bpm_check_bounded_wait": ([_I, ctypes.POINTER(_I), _P], _I),
        "bpm_batch_create": ([ctypes.c_size_t, _P, ctypes.POINTER(_P)], _I),
        "bpm_batch_submit": ([_P, _P, ctypes.POINTER(ctypes.c_uint64)], _I),
        "bpm_batch_step": ([_P, _I], _I),
        "bpm_batch_run": ([_P], _I),
        "bpm_batch_run_graph": ([_P], _I),
        "bpm_batch_poll": ([_P, ctypes.c_uint64, ctypes.POINTER(_I)], _I),
        "bpm_batch_cancel": ([_P, ctypes.c_uint64], _I),
        "bpm_batch_sync": ([_P], _I),
        "bpm_batch_info": ([_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_size_t),
                            ctypes.POINTER(_I), ctypes.POINTER(_I * 2)], _I),
        "bpm_batch_last_error": ([_P], ctypes.c_char_p),
        "bpm_batch_destroy": ([_P], None),
        "bpm_run_noalloc": ([ctypes.POINTER(Grid), _I, ctypes.POINTER(CrystalParams), _P, _P, _P,
                             ctypes.POINTER(BeamParams), _P, _P, _P, _P], _I),
        "bpm_noalloc_scratch_bytes": ([], ctypes.c_size_t),
        "bpm_noalloc_last_error": ([], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def version() -> str:
    return load().bpm_version().decode()


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _is_device(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Plan:
    """One BPM problem (crystal + pulse, n_channels frequency channels) on one GPU."""

    def __init__(self, dims, nx, ny, nz, dx, dy, dz, n_channels, stream=None, zassenhaus=1,
                 split_order=1):
        self._L = load()
        self.dims, self.nx, self.ny, self.nz = int(dims), int(nx), int(ny), int(nz)
        self.n_channels = int(n_channels)
        self.n_time = self.n_channels  # rows of the time response
        self.plane = self.nx * (self.ny if self.dims == 3 else 1)
        g = Grid(self.dims, self.nx, self.ny if self.dims == 3 else 1, self.nz, float(dx),
                 float(dy), float(dz), int(split_order), int(zassenhaus))
        h = _P()
        self._keep = []
        self._h = None
        st = self._L.bpm_plan_create(ctypes.byref(g), self.n_channels, _stream_handle(stream),
                                     ctypes.byref(h))
        if st != 0:
            raise BpmError(st, self._L.bpm_last_error(None).decode())
        self._h = h

    # -- helpers
    def _check(self, st):
        if st != 0:
            raise BpmError(st, self._L.bpm_last_error(self._h).decode())

    def close(self):
        if self._h is not None:
            self._L.bpm_plan_destroy(self._h)
            self._h = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API
    def set_crystal(self, chi0, chih, chihb, theta_B, lambda_B, x_surface, thickness, u=None):
        if u is not None and not _is_device(u):
            u = np.ascontiguousarray(u, dtype=np.float64)
            if u.size != self.nz * self.plane:
                raise ValueError("u must hold nz * ny * nx float64 values")
        chi0, chih, chihb = complex(chi0), complex(chih), complex(chihb)
        self._check(self._L.bpm_set_crystal(
            self._h, chi0.real, chi0.imag, chih.real, chih.imag, chihb.real, chihb.imag,
            float(theta_B), float(lambda_B), float(x_surface), float(thickness), _ptr(u),
            1 if _is_device(u) else 0))
        if _is_device(u):
            self._keep = [u]

    def set_crystal_shape(self, mask):
        """A crystal of any shape: mask [nz][ny][nx] (2D: [nz][nx]), nonzero =
        crystal cell, as a host array or a device tensor of one byte per cell;
        None returns to the crystal's boundaries (bpm_set_crystal_shape)."""
        if mask is None:
            self._check(self._L.bpm_set_crystal_shape(self._h, None, 0))
            return
        cells = self.nz * self.plane
        if _is_device(mask):
            if mask.numel() != cells or mask.element_size() != 1 or not mask.is_contiguous():
                raise ValueError("device mask must be a contiguous byte tensor of nz*ny*nx cells")
            self._check(self._L.bpm_set_crystal_shape(self._h, _ptr(mask), 1))
            return
        m = np.ascontiguousarray((np.asarray(mask) != 0).astype(np.uint8))
        if m.size != cells:
            raise ValueError("mask must hold nz * ny * nx cells")
        self._check(self._L.bpm_set_crystal_shape(self._h, _ptr(m), 0))

    def set_geometry(self, tan_psi=0.0, z_begin=-np.inf, z_end=np.inf):
        self._check(self._L.bpm_set_geometry(self._h, float(tan_psi), float(z_begin),
                                             float(z_end)))

    def set_pulse(self, omega, S, theta_i, x0, w0, zx=0.0, zR=1.0):
        omega = np.ascontiguousarray(omega, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.complex128)
        if omega.size != self.n_channels or S.size != self.n_channels:
            raise ValueError("omega and S need one entry per channel")
        self._check(self._L.bpm_set_pulse(self._h, _ptr(omega), _ptr(S), float(theta_i),
                                          float(x0), float(w0), float(zx), float(zR)))

    def set_fields(self, e0, eh, z_step: int):
        dev = _is_device(e0)
        if not dev:
            e0 = np.ascontiguousarray(e0, dtype=np.complex64)
            eh = np.ascontiguousarray(eh, dtype=np.complex64)
        self._check(self._L.bpm_set_fields(self._h, _ptr(e0), _ptr(eh), int(z_step),
                                           1 if dev else 0))

    def run(self, n_steps: int | None = None):
        self._check(self._L.bpm_run(self._h, self.nz if n_steps is None else int(n_steps)))

    def sync(self):
        self._check(self._L.bpm_sync(self._h))

    def set_stream(self, stream):
        self._check(self._L.bpm_set_stream(self._h, _stream_handle(stream)))

    def set_channel_shard(self, first: int, n_total: int, d_omega: float):
        """This plan holds channels first .. first + n_channels - 1 of a pulse of
        n_total channels spaced d_omega: its time response (n_total rows) and
        R_int become this shard's parts of the sums (bpm_set_channel_shard)."""
        self._check(self._L.bpm_set_channel_shard(self._h, int(first), int(n_total),
                                                  float(d_omega)))
        self.n_time = int(n_total)

    def fetch(self, which: int, out=None):
        shape = (self.n_time if which == BPM_FIELD_EH_TIME else self.n_channels, self.plane)
        if out is None:
            dt = np.complex128 if which == BPM_FIELD_EH_TIME else np.complex64
            out = np.empty(shape, dt)
        nbytes = out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes
        self._check(self._L.bpm_fetch_fields(self._h, int(which), _ptr(out), nbytes,
                                             1 if _is_device(out) else 0))
        return out

    def e0(self):
        return self.fetch(BPM_FIELD_E0)

    def eh(self):
        return self.fetch(BPM_FIELD_EH)

    def eh_time(self):
        return self.fetch(BPM_FIELD_EH_TIME)

    def reflectivity(self):
        R = np.empty(self.n_channels, np.float64)
        T = np.empty(self.n_channels, np.float64)
        rint = ctypes.c_double()
        self._check(self._L.bpm_fetch_reflectivity(self._h, _ptr(R), _ptr(T), ctypes.byref(rint)))
        return R, T, rint.value

    def set_timing(self, enable: bool = True):
        self._check(self._L.bpm_set_timing(self._h, 1 if enable else 0))

    def stats(self) -> dict:
        s = Stats()
        self._check(self._L.bpm_get_stats(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def launch(self) -> dict:
        """The plan's launch form (form, channels_per_block, row_threads)."""
        f = Launch()
        self._check(self._L.bpm_get_launch(self._h, ctypes.byref(f)))
        d = f.as_dict()
        d.pop("ms")
        return d

    def set_launch(self, form=None, channels_per_block=None, row_threads=None):
        """Force a launch form for later runs (unspecified fields keep their value)."""
        cur = self.launch()
        f = Launch(int(cur["form"] if form is None else form),
                   int(cur["channels_per_block"] if channels_per_block is None
                       else channels_per_block),
                   int(cur["row_threads"] if row_threads is None else row_threads), 0.0)
        self._check(self._L.bpm_set_launch(self._h, ctypes.byref(f)))


def tune(dims, nx, ny, dx, dy, dz, n_channels, split_order=1, zassenhaus=1, steps=16):
    """Autotune the launch form of a plan shape (C++ tuner, see bpm_tune): times
    every form on a scratch plan and keeps the fastest for later plans of this
    shape.  Returns (best, all) as dicts with the median time in ms."""
    L = load()
    g = Grid(int(dims), int(nx), int(ny) if int(dims) == 3 else 1, int(steps), float(dx),
             float(dy), float(dz), int(split_order), int(zassenhaus))
    best = Launch()
    arr = (Launch * 8)()
    n = _I(0)
    st = L.bpm_tune(ctypes.byref(g), int(n_channels), int(steps), ctypes.byref(best), arr, 8,
                    ctypes.byref(n))
    if st != 0:
        raise BpmError(st, L.bpm_last_error(None).decode())
    return best.as_dict(), [arr[i].as_dict() for i in range(n.value)]


def tune_save(path: str):
    L = load()
    if L.bpm_tune_save(os.fsencode(path)) != 0:
        raise BpmError(1, L.bpm_last_error(None).decode())


def tune_load(path: str) -> int:
    L = load()
    n = _I(0)
    if L.bpm_tune_load(os.fsencode(path), ctypes.byref(n)) != 0:
        raise BpmError(1, L.bpm_last_error(None).decode())
    return n.value


def tune_clear():
    load().bpm_tune_clear()


def plan_from_workload(w, stream=None, u=None) -> Plan:
    """Create a plan and load the crystal and the pulse of a workload record.
    u overrides w.u (e.g. with a device tensor)."""
    p = Plan(w.dims, w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.n_ch, stream=stream,
             zassenhaus=w.zassenhaus, split_order=getattr(w, "split_order", 1))
    geo = (getattr(w, "tan_psi", 0.0), getattr(w, "z_begin", -np.inf), getattr(w, "z_end", np.inf))
    if geo != (0.0, -np.inf, np.inf):
        p.set_geometry(*geo)
    if getattr(w, "mask", None) is not None:
        p.set_crystal_shape(w.mask)
    p.set_crystal(w.chi0, w.chih, w.chihb, w.theta_B, w.lambda_B, w.x_surface, w.thickness,
                  u=w.u if u is None else u)
    p.set_pulse(w.omega, w.S, w.theta_i, w.x0, w.w0, w.zx, w.zR)
    return p


def plan_bytes(dims, nx, ny, nz, n_channels, host_u=False) -> int:
    """Device bytes a plan allocates (admission by device memory)."""
    g = Grid(int(dims), int(nx), int(ny) if int(dims) == 3 else 1, int(nz), 1.0, 1.0, 1.0, 1, 1)
    return int(load().bpm_plan_bytes(ctypes.byref(g), int(n_channels), 1 if host_u else 0))


class Batch:
    """Many plans marched by one persistent work-queue launch per round
    (continuous batching: plans submitted between rounds join the next one)."""

    def __init__(self, hbm_budget_bytes: int = 0, stream=None):
        self._L = load()
        h = _P()
        self._h = None
        st = self._L.bpm_batch_create(int(hbm_budget_bytes), _stream_handle(stream),
                                      ctypes.byref(h))
        if st != 0:
            raise BpmError(st, self._L.bpm_batch_last_error(None).decode())
        self._h = h

    def _check(self, st):
        if st != 0:
            raise BpmError(st, self._L.bpm_batch_last_error(self._h).decode())

    def submit(self, plan: Plan) -> int:
        """Admit a plan; raises BpmError with status 2 (OOM) if the budget is full."""
        t = ctypes.c_uint64()
        self._check(self._L.bpm_batch_submit(self._h, plan._h, ctypes.byref(t)))
        return int(t.value)

    def try_submit(self, plan: Plan):
        t = ctypes.c_uint64()
        st = self._L.bpm_batch_submit(self._h, plan._h, ctypes.byref(t))
        if st == 2:
            return None
        self._check(st)
        return int(t.value)

    def step(self, chunk_steps: int):
        self._check(self._L.bpm_batch_step(self._h, int(chunk_steps)))

    def run(self):
        self._check(self._L.bpm_batch_run(self._h))

    def set_max_blocks(self, n: int):
        self._check(self._L.bpm_batch_set_max_blocks(self._h, int(n)))

    def graph_kernels(self) -> int:
        """Kernel launches in one replay of the captured graph."""
        n = ctypes.c_int(0)
        self._check(self._L.bpm_batch_graph_kernels(self._h, ctypes.byref(n)))
        return n.value

    def pending(self) -> int:
        """Rounds enqueued whose kernels have not finished yet."""
        n = ctypes.c_int(0)
        self._check(self._L.bpm_batch_pending(self._h, ctypes.byref(n)))
        return n.value

    def run_graph(self):
        self._check(self._L.bpm_batch_run_graph(self._h))

    def poll(self, ticket: int) -> bool:
        d = _I()
        self._check(self._L.bpm_batch_poll(self._h, ctypes.c_uint64(ticket), ctypes.byref(d)))
        return bool(d.value)

    def cancel(self, ticket: int):
        self._check(self._L.bpm_batch_cancel(self._h, ctypes.c_uint64(ticket)))

    def sync(self):
        self._check(self._L.bpm_batch_sync(self._h))

    def info(self) -> dict:
        a, r = _I(), _I()
        u = ctypes.c_size_t()
        it = (_I * 2)()
        self._check(self._L.bpm_batch_info(self._h, ctypes.byref(a), ctypes.byref(u),
                                           ctypes.byref(r), ctypes.byref(it)))
        return dict(active=a.value, used_bytes=u.value, rounds=r.value,
                    last_items=(it[0], it[1]))

    def close(self):
        if self._h is not None:
            self._L.bpm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_noalloc(w, e0_out, eh_out, refl_out, u_dev=None, stream=None):
    """Allocation-free single-instance run (bpm_run_noalloc) of a workload record.

    e0_out, eh_out: device complex64 [n_ch, nx]; refl_out: device float64 [n_ch];
    u_dev: device float64 [nz, nx] displacement or None.  For callers that must
    not allocate device memory while they run (see include/bpm.h).

    The C call takes no buffer sizes, so every tensor is checked here (CUDA,
    dtype, contiguous, element count) and a mismatch raises BpmError
    (INVALID_ARG) before anything is launched."""
    import torch
    n_ch, nx, nz = int(w.n_ch), int(w.nx), int(w.nz)

    def need(name, t, dtype, numel):
        ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype
              and t.is_contiguous() and t.numel() == numel)
        if not ok:
            got = (f"{t.device} {t.dtype} {tuple(t.shape)} contiguous={t.is_contiguous()}"
                   if isinstance(t, torch.Tensor) else type(t).__name__)
            raise BpmError(1, f"run_noalloc: {name} must be a contiguous CUDA {dtype} tensor of "
                              f"{numel} elements, got {got}")

    need("e0_out", e0_out, torch.complex64, n_ch * nx)
    need("eh_out", eh_out, torch.complex64, n_ch * nx)
    need("refl_out", refl_out, torch.float64, n_ch)
    if u_dev is not None:
        need("u_dev", u_dev, torch.float64, nz * nx)
    L = load()
    g = Grid(2, int(w.nx), 1, int(w.nz), float(w.dx), 0.0, float(w.dz), 1, int(w.zassenhaus))
    chi0, chih, chihb = complex(w.chi0), complex(w.chih), complex(w.chihb)
    c = CrystalParams(chi0.real, chi0.imag, chih.real, chih.imag, chihb.real, chihb.imag,
                      float(w.theta_B), float(w.lambda_B), float(w.x_surface), float(w.thickness))
    b = BeamParams(float(w.theta_i), float(w.x0), float(w.w0), float(w.zx), float(w.zR))
    omega = np.ascontiguousarray(w.omega, dtype=np.float64)
    S = np.ascontiguousarray(w.S, dtype=np.complex128)
    st = L.bpm_run_noalloc(ctypes.byref(g), int(w.n_ch), ctypes.byref(c), _ptr(u_dev),
                           _ptr(omega), _ptr(S), ctypes.byref(b), _ptr(e0_out), _ptr(eh_out),
                           _ptr(refl_out), _stream_handle(stream))
    if st != 0:
        raise BpmError(st, L.bpm_noalloc_last_error().decode())


BPM_PEAK_FP32, BPM_PEAK_FP64 = 0, 1


def measure_peak(kind: int = BPM_PEAK_FP32, iters: int = 1 << 16, stream=None):
    """One launch of FMA chains on every SM (bpm_measure_peak): (flop/s, ms)."""
    L = load()
    rate, ms = ctypes.c_double(), ctypes.c_float()
    st = L.bpm_measure_peak(int(kind), int(iters), ctypes.byref(rate), ctypes.byref(ms),
                            _stream_handle(stream))
    if st != 0:
        raise BpmError(st, "bpm_measure_peak failed")
    return rate.value, ms.value


def check_bounded_wait(poll_limit: int = 1 << 12, stream=None) -> bool:
    """Make one bounded bulk-copy wait run out (bpm_check_bounded_wait): True
    when it gave up and recorded the timeout status, as designed."""
    L = load()
    gave_up = ctypes.c_int()
    st = L.bpm_check_bounded_wait(int(poll_limit), ctypes.byref(gave_up), _stream_handle(stream))
    if st != 0:
        raise BpmError(st, "bpm_check_bounded_wait failed")
    return gave_up.value == 1
