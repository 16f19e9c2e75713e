"""Seeded synthetic inputs for the two-beam BPM (inputs only, no method arithmetic).

Every workload is a plain record of physical inputs: the grid, the crystal
(susceptibilities, Bragg angle, wavelength, slab surface and thickness, the
displacement field u in metres), and the incident pulse (channel angular
frequencies, complex spectral amplitudes, beam geometry).  Both the CUDA path
and the CPU oracle take these records; neither the propagators, the coupling
coefficients, the deformation phase nor the fields are computed here.

The common geometry follows the paper's diamond C*(400) case at 9.831 keV
(Bragg angle 45 degrees, Section 3 "Stationary problems"): theta_B = 45 deg,
lambda_B = 1.26116 Angstrom, chi0 = -1.0e-5 + 1.0e-8 i,
chi_h = chi_hbar = -4.0e-6 + 0.5e-8 i, theta_i = theta_B, dx = dz = 0.5 um.

Channel grid: relative detunings eps_i = eps_c + (i - n/2) * 10 eps_D / n
around the centre of the reflection band eps_c = -Re(chi0)/(2 sin^2 theta_B)
with the Darwin width eps_D = |chi_h|/sin^2 theta_B (a +-5 Darwin-width band);
omega_i = omega_B (1 + eps_i).  Spectral amplitude of the Gaussian pulse
(Eq. ref:tdp, negative exponent, t0 = 0): S_i = exp(-(eps_i-eps_c)^2/(2 s^2)),
s = 1.5 eps_D.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

C_LIGHT = 299792458.0
THETA_B = math.radians(45.0)
LAMBDA_B = 1.26116e-10
D_HKL = LAMBDA_B / (2.0 * math.sin(THETA_B))  # 0.8918 Angstrom
CHI0 = complex(-1.0e-5, 1.0e-8)
CHIH = complex(-4.0e-6, 0.5e-8)


@dataclass
class Workload:
    name: str
    dims: int
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    chi0: complex
    chih: complex
    chihb: complex
    theta_B: float
    lambda_B: float
    x_surface: float
    thickness: float
    u: np.ndarray | None  # [nz][nx] (2D) or [nz][ny][nx] (3D), float64 metres
    omega: np.ndarray  # [n_ch] rad/s
    S: np.ndarray  # [n_ch] complex128
    theta_i: float
    x0: float
    w0: float
    zx: float = 0.0
    zR: float = 1.0
    zassenhaus: int = 1
    meta: dict = field(default_factory=dict)
    split_order: int = 1  # 1: first-order splitting; 2: Strang
    # crystal shape: entrance surface x = x_surface + z tan_psi, crystal in z_begin <= z < z_end
    tan_psi: float = 0.0
    z_begin: float = -math.inf
    z_end: float = math.inf
    # an arbitrary crystal shape: [nz][nx] (2D) or [nz][ny][nx] (3D), nonzero =
    # crystal; replaces the boundaries above when given
    mask: np.ndarray | None = None

    @property
    def n_ch(self) -> int:
        return int(np.asarray(self.omega).size)

    @property
    def plane(self) -> int:
        return self.nx * (self.ny if self.dims == 3 else 1)

    @property
    def cell_updates(self) -> int:
        return self.n_ch * self.plane * self.nz

    def subset(self, channels) -> "Workload":
        idx = np.asarray(channels, dtype=np.int64)
        return replace(self, omega=np.asarray(self.omega)[idx].copy(),
                       S=np.asarray(self.S)[idx].copy())


def omega_bragg(lambda_b: float = LAMBDA_B) -> float:
    return 2.0 * math.pi * C_LIGHT / lambda_b


def band(n_ch: int, chi0=CHI0, chih=CHIH, theta_b=THETA_B, lambda_b=LAMBDA_B,
         span_darwin: float = 10.0, sigma_darwin: float = 1.5):
    """Channel frequencies over +-span/2 Darwin widths and the pulse amplitudes."""
    s2 = math.sin(theta_b) ** 2
    eps_d = abs(chih) / s2
    eps_c = -chi0.real / (2.0 * s2)
    i = np.arange(n_ch, dtype=np.float64)
    eps = eps_c + (i - n_ch // 2) * span_darwin * eps_d / n_ch
    omega = omega_bragg(lambda_b) * (1.0 + eps)
    S = np.exp(-((eps - eps_c) ** 2) / (2.0 * (sigma_darwin * eps_d) ** 2)).astype(np.complex128)
    return omega, S


def _slab(first_cell: int, n_cells: int, dx: float):
    # surfaces on half-cell boundaries so that no grid point sits on one
    return (first_cell - 0.5) * dx, n_cells * dx


def tiny(n_ch: int = 64) -> Workload:
    """Undeformed symmetric Bragg crystal, Nx=256, 200 steps, 64 channels."""
    dx = 0.5e-6
    xs, d = _slab(100, 50, dx)
    omega, S = band(n_ch)
    return Workload("tiny-2d-nx256-nz200-ch64", 2, 256, 1, 200, dx, 0.0, dx, CHI0, CHIH, CHIH,
                    THETA_B, LAMBDA_B, xs, d, None, omega, S, THETA_B, 40 * dx, 20 * dx)


def thermal_bump_2d(nx, nz, dx, dz, x_surface, amp, width):
    """u(x, z) = A exp(-x'^2/w^2) (z/Z)^2, x' = depth below the entrance surface."""
    x = np.arange(nx, dtype=np.float64) * dx
    xp = x - x_surface
    z = np.arange(nz, dtype=np.float64) * dz
    Z = nz * dz
    return amp * np.exp(-(xp[None, :] ** 2) / width ** 2) * (z[:, None] / Z) ** 2


def deformed(n_ch: int = 1024, nx: int = 4096, nz: int = 2000, seed: int = 2) -> Workload:
    """Thermal-bump deformed crystal: Nx=4096, 2000 steps, 1024 channels."""
    rng = np.random.default_rng(seed)
    dx = 0.5e-6
    s = nx / 4096.0
    xs, d = _slab(int(800 * s), int(400 * s), dx)
    amp = rng.uniform(0.0, 0.5) * D_HKL
    width = rng.uniform(20e-6, 200e-6)
    u = thermal_bump_2d(nx, nz, dx, dx, xs, amp, width)
    omega, S = band(n_ch)
    return Workload(f"deformed-2d-nx{nx}-nz{nz}-ch{n_ch}", 2, nx, 1, nz, dx, 0.0, dx, CHI0, CHIH,
                    CHIH, THETA_B, LAMBDA_B, xs, d, u, omega, S, THETA_B, int(400 * s) * dx,
                    int(40 * s) * dx, meta=dict(A=amp, w=width, seed=seed))


def _strain_field(kind, rng, nx, nz, dx, dz, xs, d):
    x = np.arange(nx, dtype=np.float64) * dx
    z = np.arange(nz, dtype=np.float64) * dz
    Z = nz * dz
    if kind == "perfect":
        return None, {}
    if kind == "bent":
        R = rng.uniform(1.0, 50.0)
        u = np.broadcast_to(-((z - Z / 2) ** 2) / (2.0 * R), (nx, nz)).T.copy()
        return u, dict(R=R)
    # random smooth strain: sum of 8 Gaussians in (depth, z), each separable
    xp = x - xs
    u = np.zeros((nz, nx))
    L = nx * dx
    for _ in range(8):
        a = rng.uniform(-0.5, 0.5) * D_HKL
        cx = rng.uniform(0.0, d)
        cz = rng.uniform(0.0, Z)
        wx = rng.uniform(L / 32, L / 4)
        wz = rng.uniform(L / 32, L / 4)
        u += a * np.outer(np.exp(-((z - cz) ** 2) / wz ** 2), np.exp(-((xp - cx) ** 2) / wx ** 2))
    return u, {}


def mixed_instance(rng, nx=None, nz=None, n_ch=None, kind=None, idx=0) -> Workload:
    """One instance of the uneven batch: Nx in {1024..8192}, 500-4000 steps,
    128-1024 channels (powers of two), perfect / bent / random-strain crystal."""
    nx = int(rng.choice([1024, 2048, 4096, 8192])) if nx is None else nx
    nz = int(rng.integers(500, 4001)) if nz is None else nz
    n_ch = int(rng.choice([128, 256, 512, 1024])) if n_ch is None else n_ch
    kind = str(rng.choice(["perfect", "bent", "random"])) if kind is None else kind
    dx = 0.5e-6
    dz = min(dx, nx * dx / (2.0 * nz))
    xs, d = _slab(nx // 5, nx // 10, dx)
    u, extra = _strain_field(kind, rng, nx, nz, dx, dz, xs, d)
    omega, S = band(n_ch)
    return Workload(f"mixed{idx}-{kind}-nx{nx}-nz{nz}-ch{n_ch}", 2, nx, 1, nz, dx, 0.0, dz, CHI0,
                    CHIH, CHIH, THETA_B, LAMBDA_B, xs, d, u, omega, S, THETA_B, (nx // 10) * dx,
                    max(8, nx // 100) * dx, meta=dict(kind=kind, **extra))


def batch(n_inst: int = 64, seed: int = 3):
    """Uneven batch of instances (seeded)."""
    rng = np.random.default_rng(seed)
    return [mixed_instance(rng, idx=i) for i in range(n_inst)]


def probe(rng, idx=0) -> Workload:
    """Single-channel rocking-curve probe: Nx=512, 300 steps, incidence angle
    theta_B + U(+-5 Darwin widths)."""
    dx = 0.5e-6
    nx, nz = 512, 300
    xs, d = _slab(nx // 4, nx // 8, dx)
    s2 = math.sin(THETA_B) ** 2
    eps_d = abs(CHIH) / s2
    dth = rng.uniform(-5.0, 5.0) * eps_d * math.tan(THETA_B)
    omega = np.array([omega_bragg()], np.float64)
    S = np.ones(1, np.complex128)
    return Workload(f"probe{idx}-nx512-nz300", 2, nx, 1, nz, dx, 0.0, dx, CHI0, CHIH, CHIH,
                    THETA_B, LAMBDA_B, xs, d, None, omega, S, THETA_B + dth, (nx // 10) * dx,
                    16 * dx, meta=dict(dtheta=dth))


def serving_stream(n_req: int = 10000, seed: int = 4, probe_frac: float = 0.8):
    """Request mix: probe_frac rocking-curve probes, the rest uneven-batch instances.
    Returns the list of workloads (arrival times are drawn by the server)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_req):
        if rng.uniform() < probe_frac:
            out.append(probe(rng, idx=i))
        else:
            out.append(mixed_instance(rng, idx=i))
    return out


def thermal_bump_3d(nx, ny, nz, dx, dy, dz, x_surface, amp, wx, wy):
    x = np.arange(nx, dtype=np.float64) * dx
    y = (np.arange(ny, dtype=np.float64) - ny // 2) * dy
    z = np.arange(nz, dtype=np.float64) * dz
    Z = nz * dz
    xy = np.exp(-((x - x_surface)[None, :] ** 2) / wx ** 2 - (y[:, None] ** 2) / wy ** 2)
    return amp * xy[None, :, :] * ((z / Z) ** 2)[:, None, None]


def large_3d(n_ch: int = 128, nx: int = 512, ny: int = 512, nz: int = 1000, seed: int = 5,
             with_u: bool = True) -> Workload:
    """3D (x, y, z): 512 x 512 transverse, 1000 steps of 0.25 um, 128 channels,
    120 um slab, thermal bump u(x, y, z)."""
    rng = np.random.default_rng(seed)
    dx = dy = 1.0e-6
    dz = 0.25e-6
    s = nx / 512.0
    xs, d = _slab(int(160 * s), int(120 * s), dx)
    amp = rng.uniform(0.0, 0.5) * D_HKL
    wx = rng.uniform(20e-6, 100e-6)
    wy = rng.uniform(20e-6, 100e-6)
    u = thermal_bump_3d(nx, ny, nz, dx, dy, dz, xs, amp, wx, wy) if with_u else None
    omega, S = band(n_ch)
    return Workload(f"large-3d-{nx}x{ny}-nz{nz}-ch{n_ch}", 3, nx, ny, nz, dx, dy, dz, CHI0, CHIH,
                    CHIH, THETA_B, LAMBDA_B, xs, d, u, omega, S, THETA_B, int(80 * s) * dx,
                    int(40 * s) * dx, meta=dict(A=amp, wx=wx, wy=wy, seed=seed))


def strain_gradient(B: float = 0.25, beta_ratio: float = 4.7326, depth_um: float = 140.0,
                    nx: int = 4096, dx: float = 0.25e-6, dz: float = 0.5e-6,
                    z_end_um: float = 900.0, w0_um: float = 20.0) -> Workload:
    """Constant strain gradient in a symmetric Bragg crystal (Section 3.2,
    "Deformed crystals"): Si(444) at 17 keV (lambda = 0.72932 A, d = a/sqrt(48),
    a = 5.43102 A), absorption and refraction off (chi0 = 0, chi_h real), and
    displacement u = B x'^2 along h (x' = depth below the entrance surface),
    the reading of the garbled Eq. Authier2 that reproduces the strain-gradient
    parameter beta = 4 B sin^2(theta_B) tan(theta_B)/|chi_h| (Eq. Yan).
    |chi_h| is taken from the paper's printed ratio beta/beta_c, with
    beta_c = pi/(2 Lambda0) and Lambda0 = lambda cos(theta_B)/|chi_h|:
    beta/beta_c = 8 B lambda sin^3(theta_B)/(pi |chi_h|^2).

    A single channel at the Bragg wavelength enters at theta_B + 2 B x_r
    tan(theta_B), so that the local Bragg condition is met x_r = depth_um below
    the surface, far from both faces of a crystal of thickness x_r + 80 um.
    The beam starts 60 um in front of the surface; after z_end the transmitted
    branch has left through the back face and the reflected one through the
    front face, neither wrapping around the periodic x window.
    meta: B, beta_ratio, the Landau-Zener fraction exp(-2 pi / beta_ratio) of
    the new (transmitted) branch, and the x of both faces."""
    lam = 0.72932e-10
    theta_b = math.asin(lam / (2.0 * 5.43102e-10 / math.sqrt(48.0)))
    chih = -math.sqrt(8.0 * B * lam * math.sin(theta_b) ** 3 / (math.pi * beta_ratio))
    nz = int(round(z_end_um * 1e-6 / dz))
    xs = 300e-6 + 0.5 * dx
    thickness = (depth_um + 80.0) * 1e-6
    x = np.arange(nx, dtype=np.float64) * dx
    depth = np.clip(x - xs, 0.0, None)
    u = np.tile(B * depth ** 2, (nz, 1))
    theta_i = theta_b + 2.0 * B * depth_um * 1e-6 * math.tan(theta_b)
    omega = np.array([2.0 * math.pi * C_LIGHT / lam])
    return Workload(f"strain-gradient-B{B}", 2, nx, 1, nz, dx, 0.0, dz, 0j, complex(chih, 0.0),
                    complex(chih, 0.0), theta_b, lam, xs, thickness, u, omega,
                    np.ones(1, np.complex128), theta_i, xs - 60e-6, w0_um * 1e-6,
                    meta=dict(B=B, beta_ratio=beta_ratio,
                              interbranch=math.exp(-2.0 * math.pi / beta_ratio),
                              x_front=xs, x_back=xs + thickness))
