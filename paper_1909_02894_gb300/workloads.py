"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: metric fields g00, g11, g22 on the grid, the initial
two-component spinor and the run parameters. It holds none of the method's arithmetic
(no transforms, coefficients, time stepping or observables), so both the CUDA path
and the CPU oracle can take their inputs from here.

Grid convention (Sec. 5): x_j = -a + j*h with h = 2a/N, j = 0..N-1; arrays are
[ny][nx] with x fastest; a spinor is [2][ny][nx] complex128.

The paper prints no dataset; its tests are analytic initial-value problems (Sec. 6).
The recipes below stand in for its convergence test (Experiment 3, a Gaussian packet
in a smooth static metric) and its strained-graphene tests (Sec. 6.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

CONN_COVARIANT = 0
CONN_PAPER_2D = 1
CONN_NONE = 2


@dataclass
class Workload:
    """One simulation: grid, metric fields, mass, c, absorbing layer, packet, time step."""

    name: str
    nx: int
    ny: int
    ax: float
    ay: float
    g00: Optional[np.ndarray]
    g11: Optional[np.ndarray]
    g22: Optional[np.ndarray]
    mass: float
    c: float
    pml_width_x: int
    pml_width_y: int
    pml_type: int
    sigma0: float
    theta: float
    psi0: np.ndarray  # complex128 [2][ny][nx]
    dt: float
    steps: int
    conn: int = CONN_COVARIANT
    meta: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return self.nx * self.ny


def grid_1d(n: int, a: float) -> np.ndarray:
    """x_j = -a + j*2a/n (Sec. 5)."""
    return -a + np.arange(n, dtype=np.float64) * (2.0 * a / n)


def mesh(nx: int, ny: int, ax: float, ay: float):
    x = grid_1d(nx, ax)
    y = grid_1d(ny, ay)
    return np.meshgrid(x, y, indexing="xy")  # X[j][i] = x_i, Y[j][i] = y_j


def gaussian(X, Y, cx, cy, w):
    """G(x; c, w) = exp(-|x - c|^2 / (2 w^2))."""
    return np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * w * w))


def wave_packet(nx, ny, ax, ay, width, k0, x0=(0.0, 0.0), phase=0.0) -> np.ndarray:
    """Upper-component Gaussian packet A exp(-|x-x0|^2/(2w^2) + i k0.x + i phase).

    A = 1/(w sqrt(pi)) makes the continuous L2 norm one.
    """
    X, Y = mesh(nx, ny, ax, ay)
    amp = 1.0 / (width * np.sqrt(np.pi))
    psi = np.zeros((2, ny, nx), dtype=np.complex128)
    psi[0] = amp * np.exp(
        -((X - x0[0]) ** 2 + (Y - x0[1]) ** 2) / (2.0 * width * width)
        + 1j * (k0[0] * X + k0[1] * Y)
        + 1j * phase
    )
    return psi


def random_state(nx, ny, seed) -> np.ndarray:
    """Seeded complex white noise, for brute-force and linearity checks."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((2, ny, nx)) + 1j * rng.standard_normal((2, ny, nx))


def plane_waves(nx, ny, ax, ay, modes) -> np.ndarray:
    """Sum of plane waves; modes = [(qx, qy, (A1, A2))] with FFT indices qx, qy.

    psi(x_j, y_l) = sum A exp(i xi_x (x_j + ax)) exp(i xi_y (y_l + ay)) where
    xi = p pi / a and p is q mapped into [-N/2, N/2).
    """
    X, Y = mesh(nx, ny, ax, ay)
    psi = np.zeros((2, ny, nx), dtype=np.complex128)
    for qx, qy, amps in modes:
        px = qx if qx < nx // 2 else qx - nx
        py = qy if qy < ny // 2 else qy - ny
        e = np.exp(1j * (px * np.pi / ax) * (X + ax) + 1j * (py * np.pi / ay) * (Y + ay))
        psi[0] += amps[0] * e
        psi[1] += amps[1] * e
    return psi


# ---------------------------------------------------------------------------------
# Workload recipes (seeded). Sizes are the paper-shaped configurations; "scale"
# variants keep the same recipe at a smaller grid for the oracle.
# ---------------------------------------------------------------------------------

def plain_128(n: int = 128, flat: bool = False, steps: int = 200, seed: int = 1909) -> Workload:
    """Plain single instance: 2-spinor on an n x n periodic grid, domain [-20,20]^2,
    c=1, m=0, g00=1, g11=g22=1+0.1 exp(-|x|^2/9) (flat twin: g11=g22=1), packet of
    width 2 with k0=(2,0), upper component, seeded phase; no absorbing layer; dt=0.01."""
    rng = np.random.default_rng(seed)
    phase = 2.0 * np.pi * rng.uniform()
    a = 20.0
    X, Y = mesh(n, n, a, a)
    g00 = np.ones((n, n))
    if flat:
        g11 = np.ones((n, n))
    else:
        g11 = 1.0 + 0.1 * np.exp(-(X ** 2 + Y ** 2) / 9.0)
    g22 = g11.copy()
    psi = wave_packet(n, n, a, a, 2.0, (2.0, 0.0), phase=phase)
    return Workload(
        name=f"plain-{n}^2" + ("-flat" if flat else ""), nx=n, ny=n, ax=a, ay=a,
        g00=g00, g11=g11, g22=g22, mass=0.0, c=1.0,
        pml_width_x=0, pml_width_y=0, pml_type=1, sigma0=1.0, theta=0.0,
        psi0=psi, dt=0.01, steps=steps,
    )


def graphene_strained(n: int = 1024, steps: int = 5000, seed: int = 1910,
                      pml: Optional[int] = None) -> Workload:
    """Strained-graphene single instance. n=1024 is the paper-shaped size: domain
    [-100,100]^2, m=0, c=1, uniaxial pre-strain 0.1 along x times a Gaussian
    out-of-plane bump (amplitude 0.2, width 15): g11=(1.1)(1+0.2G), g22=1+0.2G, g00=1;
    absorbing layer 64 points (type I, sigma0=1, theta=0); packet width 8,
    k0=(1.5,0.5); dt=0.05. Smaller n keeps h and scales the domain."""
    rng = np.random.default_rng(seed)
    phase = 2.0 * np.pi * rng.uniform()
    h = 200.0 / 1024.0
    a = n * h / 2.0
    X, Y = mesh(n, n, a, a)
    bump = 0.2 * gaussian(X, Y, 0.0, 0.0, 15.0)
    g00 = np.ones((n, n))
    g11 = 1.1 * (1.0 + bump)
    g22 = 1.0 + bump
    width = max(4, (64 * n) // 1024) if pml is None else pml
    psi = wave_packet(n, n, a, a, min(8.0, a / 6.0), (1.5, 0.5), phase=phase)
    return Workload(
        name=f"graphene-{n}^2", nx=n, ny=n, ax=a, ay=a,
        g00=g00, g11=g11, g22=g22, mass=0.0, c=1.0,
        pml_width_x=width, pml_width_y=width, pml_type=1, sigma0=1.0, theta=0.0,
        psi0=psi, dt=0.05, steps=steps,
    )


def random_bumps_metric(n, a, nbumps, amp_range, width_range, interior, rng):
    """g11 = g22 = 1 + sum_b A_b G(x; c_b, w_b), centres uniform in [-interior, interior]^2."""
    X, Y = mesh(n, n, a, a)
    g = np.ones((n, n))
    for _ in range(nbumps):
        cx, cy = rng.uniform(-interior, interior, size=2)
        amp = rng.uniform(*amp_range)
        w = rng.uniform(*width_range)
        g += amp * gaussian(X, Y, cx, cy, w)
    return g


def large_4096(n: int = 4096, steps: int = 1000, seed: int = 1912) -> Workload:
    """Large single grid: n=4096 complex64 spinor, m=0.5, c=1, random smooth strain
    (16 Gaussian bumps, amplitudes U[0,0.15], widths U[10,40], seeded centres inside
    the absorbing layer's inner edge), absorbing layer 128 points (type I, sigma0=1),
    packet width 8, k0=(1.5,0.5), dt=0.05; h=200/1024 so a=400 at n=4096."""
    rng = np.random.default_rng(seed)
    phase = 2.0 * np.pi * rng.uniform()
    h = 200.0 / 1024.0
    a = n * h / 2.0
    width = 128 if n >= 4096 else max(4, n // 32)
    interior = a - width * h
    g = random_bumps_metric(n, a, 16, (0.0, 0.15), (10.0, 40.0), interior, rng)
    psi = wave_packet(n, n, a, a, 8.0, (1.5, 0.5), phase=phase)
    return Workload(
        name=f"large-{n}^2", nx=n, ny=n, ax=a, ay=a,
        g00=np.ones((n, n)), g11=g, g22=g.copy(), mass=0.5, c=1.0,
        pml_width_x=width, pml_width_y=width, pml_type=1, sigma0=1.0, theta=0.0,
        psi0=psi, dt=0.05, steps=steps,
    )


def batched_instance(n: int, rng: np.random.Generator, steps: int = 2000) -> Workload:
    """One instance of the uneven batch: h=0.2, a=n h/2, 4 bumps (A~U[0,0.15],
    w~U[0.05,0.2]*2a), conformal metric g00=1, absorbing layer max(8, n/16) points,
    packet width U[0.05,0.1]*2a, k0~U[-2,2]^2, centre in the inner half; dt=0.05."""
    h = 0.2
    a = n * h / 2.0
    width = max(8, n // 16)
    interior = a - width * h
    X, Y = mesh(n, n, a, a)
    g = np.ones((n, n))
    for _ in range(4):
        cx, cy = rng.uniform(-interior, interior, size=2)
        amp = rng.uniform(0.0, 0.15)
        w = rng.uniform(0.05, 0.2) * 2.0 * a
        g += amp * gaussian(X, Y, cx, cy, w)
    pw = rng.uniform(0.05, 0.1) * 2.0 * a
    k0 = rng.uniform(-2.0, 2.0, size=2)
    x0 = rng.uniform(-a / 2.0, a / 2.0, size=2)
    phase = 2.0 * np.pi * rng.uniform()
    psi = wave_packet(n, n, a, a, pw, tuple(k0), x0=tuple(x0), phase=phase)
    return Workload(
        name=f"batch-{n}^2", nx=n, ny=n, ax=a, ay=a,
        g00=np.ones((n, n)), g11=g, g22=g.copy(), mass=0.0, c=1.0,
        pml_width_x=width, pml_width_y=width, pml_type=1, sigma0=1.0, theta=0.0,
        psi0=psi, dt=0.05, steps=steps,
    )


BATCH_SIZES = (128, 256, 512, 1024)
BATCH_WEIGHTS = (0.4, 0.3, 0.2, 0.1)


def batch_sizes(count: int = 256, seed: int = 1913) -> List[int]:
    """Grid sizes of the uneven batch, drawn from {128,256,512,1024}^2 with weights
    0.4/0.3/0.2/0.1."""
    rng = np.random.default_rng(seed)
    return [int(s) for s in rng.choice(BATCH_SIZES, size=count, p=BATCH_WEIGHTS)]


def batch_mix(count: int = 256, steps: int = 2000, seed: int = 1913,
              sizes: Optional[List[int]] = None) -> List[Workload]:
    rng = np.random.default_rng(seed + 1)
    sizes = batch_sizes(count, seed) if sizes is None else sizes
    return [batched_instance(n, rng, steps) for n in sizes]


SERVE_SIZES = (256, 512, 1024, 2048)


def serve_requests(rate: float = 200.0, duration: float = 60.0, seed: int = 1914,
                   sizes=SERVE_SIZES, steps_range=(500, 5000)):
    """Poisson arrivals: list of (arrival_time_s, n, steps, instance_seed)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        n = int(rng.choice(sizes))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append((t, n, steps, int(rng.integers(0, 2 ** 31 - 1))))
    return out


def serve_instance(n: int, steps: int, seed: int) -> Workload:
    """Strained-graphene family scaled to n (h = 200/1024, bump width scaled)."""
    rng = np.random.default_rng(seed)
    h = 200.0 / 1024.0
    a = n * h / 2.0
    X, Y = mesh(n, n, a, a)
    amp = rng.uniform(0.1, 0.3)
    bw = rng.uniform(0.05, 0.1) * 2.0 * a
    bump = amp * gaussian(X, Y, 0.0, 0.0, bw)
    eps = rng.uniform(0.0, 0.15)
    width = max(8, n // 16)
    k0 = rng.uniform(-2.0, 2.0, size=2)
    psi = wave_packet(n, n, a, a, rng.uniform(0.03, 0.06) * 2.0 * a, tuple(k0),
                      phase=2.0 * np.pi * rng.uniform())
    return Workload(
        name=f"serve-{n}^2", nx=n, ny=n, ax=a, ay=a,
        g00=np.ones((n, n)), g11=(1.0 + eps) * (1.0 + bump), g22=1.0 + bump,
        mass=0.0, c=1.0, pml_width_x=width, pml_width_y=width, pml_type=1,
        sigma0=1.0, theta=0.0, psi0=psi, dt=0.05, steps=steps,
    )


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2 over both components and all points."""
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
