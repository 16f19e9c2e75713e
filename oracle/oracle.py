"""FP64 CPU oracle for the two-beam FFT BPM (arXiv:2201.08500, Section 2).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference legs of bench.py, never by the product library.  It
shares no code with the CUDA path; the heavy split-step march lives in
``bpm_oracle.c`` (plain C, FP64), the plain sums (reflectivity, the
frequency-to-time transform) are written here in numpy FP64.

Inputs are duck-typed: any object with the attributes of a workload
(dims, nx, ny, nz, dx, dy, dz, chi0, chih, chihb, theta_B, lambda_B,
x_surface, thickness, u, omega, S, theta_i, x0, w0, zx, zR, zassenhaus).

Parity status of each function (pins in tests/test_oracle_pins.py):
  fft / dft / fft2 ........ pinned (direct DFT, numpy.fft, round trip)
  bessel_j0_g1 ............ pinned (scipy.special, trapezoidal quadrature)
  channel (propagators) ... pinned (free-space Gaussian-beam closed form,
                            beam-centroid speed tan(theta_B))
  channel (a, b+-) ........ pinned (flux identity, Beer-Lambert absorption,
                            Laue pendelloesung, Bragg-slab rocking curve)
  march ................... pinned (per-mode 2x2 matrix power with the direct
                            DFT; split run; channel independence)
  deformation ............. pinned (uniform displacement leaves |fields|,
                            uniform strain equals a rescaled h)
  reflectivity ............ pinned (textbook Bragg-slab curve)
  omega_to_t .............. pinned (numpy.fft, Parseval)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bpm_oracle.c")
LIB = os.path.join(HERE, "libbpm_oracle.so")

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/libbpm_oracle.so (plain gcc)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    # no FMA contraction: mask decisions and phases round the same way on every host
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", SRC,
           "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class Problem(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("nz", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
        ("chi0_re", ctypes.c_double), ("chi0_im", ctypes.c_double),
        ("chih_re", ctypes.c_double), ("chih_im", ctypes.c_double),
        ("chihb_re", ctypes.c_double), ("chihb_im", ctypes.c_double),
        ("theta_B", ctypes.c_double), ("lambda_B", ctypes.c_double),
        ("x_surface", ctypes.c_double), ("thickness", ctypes.c_double),
        ("zassenhaus", ctypes.c_int32), ("split_order", ctypes.c_int32),
        ("theta_i", ctypes.c_double), ("x0", ctypes.c_double), ("w0", ctypes.c_double),
        ("zx", ctypes.c_double), ("zR", ctypes.c_double),
        ("tan_psi", ctypes.c_double), ("z_begin", ctypes.c_double), ("z_end", ctypes.c_double),
        ("mask", ctypes.c_void_p),
    ]


_P = ctypes.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            L.orc_dft.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int]
            L.orc_fft.argtypes = [_P, ctypes.c_int, ctypes.c_int]
            L.orc_fft2.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_bessel_j0_g1.argtypes = [_P, _P, _P]
            L.orc_channel.argtypes = [ctypes.POINTER(Problem), ctypes.c_double, _P, _P, _P, _P]
            L.orc_deformation.argtypes = [ctypes.POINTER(Problem), _P, ctypes.c_int, _P, _P]
            L.orc_incident.argtypes = [ctypes.POINTER(Problem), ctypes.c_double, _P, _P, _P]
            L.orc_march.argtypes = [ctypes.POINTER(Problem), _P, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, _P, _P]
            L.orc_run.argtypes = [ctypes.POINTER(Problem), _P, ctypes.c_int, _P, _P, ctypes.c_int,
                                  _P, _P, ctypes.c_int]
            for f in ("orc_dft", "orc_fft", "orc_fft2", "orc_bessel_j0_g1", "orc_channel",
                      "orc_deformation", "orc_incident", "orc_march", "orc_run"):
                getattr(L, f).restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def problem(w) -> Problem:
    """Build the C problem record from a workload-like object.  An optional
    w.mask ([nz][ny][nx], nonzero = crystal) replaces the geometric crystal
    boundaries; the record keeps its byte copy alive."""
    dims = int(w.dims)
    mask = getattr(w, "mask", None)
    mbytes = None
    if mask is not None:
        ny = int(w.ny) if dims == 3 else 1
        mbytes = np.ascontiguousarray((np.asarray(mask) != 0).astype(np.uint8))
        if mbytes.size != int(w.nz) * ny * int(w.nx):
            raise ValueError("mask must hold nz * ny * nx cells")
    rec = Problem(
        dims, int(w.nx), int(w.ny) if dims == 3 else 1, int(w.nz),
        float(w.dx), float(w.dy) if dims == 3 else 0.0, float(w.dz),
        complex(w.chi0).real, complex(w.chi0).imag,
        complex(w.chih).real, complex(w.chih).imag,
        complex(w.chihb).real, complex(w.chihb).imag,
        float(w.theta_B), float(w.lambda_B), float(w.x_surface), float(w.thickness),
        int(w.zassenhaus), int(getattr(w, "split_order", 1)),
        float(w.theta_i), float(w.x0), float(w.w0), float(w.zx), float(w.zR),
        float(getattr(w, "tan_psi", 0.0)), float(getattr(w, "z_begin", -np.inf)),
        float(getattr(w, "z_end", np.inf)),
        None if mbytes is None else mbytes.ctypes.data_as(ctypes.c_void_p),
    )
    rec._mask_bytes = mbytes
    return rec


def _plane(w) -> int:
    return int(w.nx) * (int(w.ny) if int(w.dims) == 3 else 1)


def _u_array(w):
    if w.u is None:
        return None
    u = np.ascontiguousarray(w.u, dtype=np.float64)
    if u.size != int(w.nz) * _plane(w):
        raise ValueError("u-field must hold nz * ny * nx values")
    return u


# --------------------------------------------------------------------------- transforms
def dft(a, sign: int = -1) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    out = np.empty_like(a)
    _check(lib().orc_dft(_ptr(a), _ptr(out), a.size, sign), "dft")
    return out


def fft(a, sign: int = -1) -> np.ndarray:
    a = np.array(a, dtype=np.complex128, copy=True)
    _check(lib().orc_fft(_ptr(a), a.size, sign), "fft")
    return a


def fft2(a, sign: int = -1) -> np.ndarray:
    a = np.array(a, dtype=np.complex128, copy=True)
    ny, nx = a.shape
    _check(lib().orc_fft2(_ptr(a), nx, ny, sign), "fft2")
    return a


def bessel_j0_g1(w2: complex):
    """J0(w) and G1(w) = 2 J1(w)/w as functions of w^2 (power series)."""
    j0 = np.zeros(1, np.complex128)
    g1 = np.zeros(1, np.complex128)
    arg = np.array([complex(w2).real, complex(w2).imag], np.float64)
    _check(lib().orc_bessel_j0_g1(_ptr(arg), _ptr(j0), _ptr(g1)), "bessel")
    return complex(j0[0]), complex(g1[0])


# --------------------------------------------------------------------------- physics pieces
def channel(w, omega: float, tables: bool = True) -> dict:
    """Per-channel scalars, coupling coefficients and tilted propagators."""
    p = problem(w)
    sc = np.zeros(5, np.float64)
    coef = np.zeros(3, np.complex128)
    shape = (_plane(w),)
    pp = np.zeros(shape, np.complex128) if tables else None
    pm = np.zeros(shape, np.complex128) if tables else None
    _check(lib().orc_channel(ctypes.byref(p), float(omega), _ptr(sc), _ptr(coef), _ptr(pp),
                             _ptr(pm)), "channel")
    return dict(k=sc[0], h=sc[1], cos_alpha=sc[2], w2=complex(sc[3], sc[4]), a=coef[0],
                bp=coef[1], bm=coef[2], pp=pp, pm=pm)


def deformation(w, z_index: int):
    p = problem(w)
    n = _plane(w)
    c = np.zeros(n, np.complex128)
    m = np.zeros(n, np.uint8)
    u = _u_array(w)
    _check(lib().orc_deformation(ctypes.byref(p), _ptr(u), int(z_index), _ptr(c), _ptr(m)),
           "deformation")
    return c, m


def incident(w, omega: float, S: complex) -> np.ndarray:
    p = problem(w)
    e0 = np.zeros(_plane(w), np.complex128)
    s = np.array([complex(S).real, complex(S).imag], np.float64)
    _check(lib().orc_incident(ctypes.byref(p), float(omega), _ptr(s), _ptr(e0), None), "incident")
    return e0


def march(w, omega: float, z_begin: int, n_steps: int, e0: np.ndarray, eh: np.ndarray):
    """Advance one channel's envelopes in place (arrays of nx*ny complex128)."""
    assert e0.dtype == np.complex128 and eh.dtype == np.complex128
    assert e0.flags.c_contiguous and eh.flags.c_contiguous
    p = problem(w)
    u = _u_array(w)
    _check(lib().orc_march(ctypes.byref(p), _ptr(u), float(omega), int(z_begin), int(n_steps),
                           _ptr(e0), _ptr(eh)), "march")


def run(w, n_steps: int | None = None, channels=None, n_threads: int | None = None):
    """Incident field + z-march for the selected channels.

    Returns (e0, eh, e0_init), each [n_sel, nx*ny] complex128."""
    omega = np.ascontiguousarray(np.asarray(w.omega, np.float64))
    S = np.ascontiguousarray(np.asarray(w.S, np.complex128))
    if channels is not None:
        idx = np.asarray(channels, dtype=np.int64)
        omega = np.ascontiguousarray(omega[idx])
        S = np.ascontiguousarray(S[idx])
    n_ch = omega.size
    n = _plane(w)
    steps = int(w.nz) if n_steps is None else int(n_steps)
    e0 = np.zeros((n_ch, n), np.complex128)
    eh = np.zeros((n_ch, n), np.complex128)
    init = np.zeros((n_ch, n), np.complex128)
    for i in range(n_ch):
        init[i] = incident(w, omega[i], S[i])
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    p = problem(w)
    u = _u_array(w)
    _check(lib().orc_run(ctypes.byref(p), _ptr(u), n_ch, _ptr(omega), _ptr(S), steps, _ptr(e0),
                         _ptr(eh), int(n_threads)), "run")
    return e0, eh, init


# --------------------------------------------------------------------------- plain sums
def reflectivity(e0_init, e0, eh):
    """R_i = sum_x |A-(Z)|^2 / sum_x |A+(0)|^2 and T_i likewise for A+(Z)."""
    inc = np.sum(np.abs(np.asarray(e0_init, np.complex128)) ** 2, axis=-1)
    R = np.sum(np.abs(np.asarray(eh, np.complex128)) ** 2, axis=-1) / inc
    T = np.sum(np.abs(np.asarray(e0, np.complex128)) ** 2, axis=-1) / inc
    return R, T


def channel_spacing(omega) -> float:
    omega = np.asarray(omega, np.float64)
    return float(omega[1] - omega[0]) if omega.size > 1 else 1.0


def integrated_reflectivity(R, omega) -> float:
    """R_int = d_omega * sum_i R_i (rectangle rule over the channel grid)."""
    return channel_spacing(omega) * float(np.sum(np.asarray(R, np.float64)))


def omega_to_t(eh, domega: float) -> np.ndarray:
    """psi_h(t_j, x) = d_omega * sum_i A-(omega_i, x) exp(-2 pi i (i - n/2) j / n).

    The text after Eq. ref:tdp sums over the channel grid with exp(-i omega t);
    relative to the centre channel i_c = n/2 and on the grid t_j = 2 pi j /
    (n d_omega) the phase is exactly 2 pi (i - i_c) j / n.  Direct FP64 sum."""
    eh = np.asarray(eh, np.complex128)
    n = eh.shape[0]
    ic = n // 2
    i = np.arange(n)
    j = np.arange(n)
    ph = np.mod(np.outer(j, i - ic), n).astype(np.float64)
    kern = np.exp(-2j * np.pi * ph / n)
    flat = eh.reshape(n, -1)
    out = domega * (kern @ flat)
    return out.reshape(eh.shape)
