"""Seeded synthetic inputs shaped like the paper's examples (numpy only).

This module holds no arithmetic of the PSTD method: it only draws Gaussian
initial pressures on the full node lattice x_j = j dx, j = 0..N per axis, and
names the workloads.  Both the CUDA path and the FP64 oracle consume what it
returns; neither side's code lives here.

Workloads (sound speed 1500 m/s, density 1000 kg/m^3, dx = 0.1 mm):
  line256_dd      1-D, N = 256, Dirichlet both ends, one Gaussian (sigma 4 dx,
                  1 Pa) at node 100, zero velocity, CFL 0.2, 2000 steps
  plane512_dx_ny  2-D, 512 x 512, Dirichlet on the x walls, Neumann on the y
                  walls, 4 Gaussians (sigma 3 dx, amplitude U[0.5, 1]) at
                  seeded uniform positions, CFL 0.3, 4000 steps
  cube256_*       3-D, 256^3, one Gaussian blob (sigma 3 dx), CFL 0.3
  cube384_dnd     3-D, 384^3, Dirichlet x / Neumann y / Dirichlet z, 4 blobs,
                  CFL 0.3, 1000 steps
  cube256_r0.4    3-D 256^3 with reflection coefficient 0.4 on every face:
                  the 64 Neumann/Dirichlet combinations of Section 5
  plane_batch     64 independent 2-D runs of seeded sizes in [64, 1024]^2
                  with random walls (each wall N or D with probability 1/2)
Blob centres are drawn uniformly in [4 sigma, L - 4 sigma] per axis so that the
field is negligible at the walls.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C0 = 1500.0
RHO0 = 1000.0
DX = 1.0e-4


@dataclass
class Blob:
    centre: tuple          # physical position per axis [m]
    sigma: float           # [m]
    amplitude: float       # [Pa]


@dataclass
class Workload:
    name: str
    ncells: tuple
    bc: tuple              # per axis (left, right), "N" or "D"
    cfl: float
    steps: int
    blobs: list = field(default_factory=list)
    dx: float = DX
    c0: float = C0
    rho0: float = RHO0
    refl: list = None      # per axis (R_left, R_right) for reflection-coefficient runs

    @property
    def ndim(self) -> int:
        return len(self.ncells)

    def factors(self):
        """Per blob, per axis: the 1-D Gaussian profile on nodes j = 0..N (FP64).

        The initial pressure is sum_b amplitude_b * prod_i factor[b][i].
        """
        out = []
        for b in self.blobs:
            term = []
            for i, n in enumerate(self.ncells):
                x = np.arange(n + 1, dtype=np.float64) * self.dx
                g = np.exp(-((x - b.centre[i]) ** 2) / (2.0 * b.sigma ** 2))
                if i == 0:
                    g = g * b.amplitude
                term.append(g)
            out.append(term)
        return out

    def p0_full(self) -> np.ndarray:
        """Initial pressure on the full node lattice, shape (N_0+1, ..., N_{d-1}+1), FP64."""
        p = np.zeros(tuple(n + 1 for n in self.ncells))
        for term in self.factors():
            t = term[0]
            for g in term[1:]:
                t = np.multiply.outer(t, g)
            p += t
        return p


def random_blobs(ncells, nblobs, sigma_cells, amp_range, seed, dx=DX):
    rng = np.random.default_rng(seed)
    sigma = sigma_cells * dx
    blobs = []
    for _ in range(nblobs):
        centre = tuple(float(rng.uniform(4 * sigma, n * dx - 4 * sigma)) for n in ncells)
        amp = float(rng.uniform(*amp_range)) if amp_range[0] != amp_range[1] else float(amp_range[0])
        blobs.append(Blob(centre, sigma, amp))
    return blobs


def line256_dd() -> Workload:
    return Workload("line256_dd", (256,), (("D", "D"),), 0.2, 2000,
                    [Blob((100 * DX,), 4 * DX, 1.0)])


def plane512_dx_ny(seed: int = 0) -> Workload:
    n = (512, 512)
    return Workload("plane512_dx_ny", n, (("D", "D"), ("N", "N")), 0.3, 4000,
                    random_blobs(n, 4, 3.0, (0.5, 1.0), seed))


def cube256(bc=(("D", "D"), ("N", "N"), ("D", "D")), seed: int = 0, steps: int = 1500) -> Workload:
    n = (256, 256, 256)
    tag = "".join(l + r for l, r in bc).lower()
    return Workload(f"cube256_{tag}", n, tuple(bc), 0.3, steps,
                    random_blobs(n, 1, 3.0, (1.0, 1.0), seed))


def cube384_dnd(seed: int = 0) -> Workload:
    n = (384, 384, 384)
    return Workload("cube384_dnd", n, (("D", "D"), ("N", "N"), ("D", "D")), 0.3, 1000,
                    random_blobs(n, 4, 3.0, (0.5, 1.0), seed))


def cube256_reflect(r: float = 0.4, seed: int = 0, steps: int = 1500) -> Workload:
    """3-D 256^3, reflection coefficient r on all six faces (64 wall combinations)."""
    w = cube256(seed=seed, steps=steps)
    w.name = f"cube256_r{r:g}"
    w.refl = [(r, r)] * 3
    w.bc = (("N", "N"),) * 3     # placeholder: the 64 combinations replace it
    return w


def plane_batch(n: int = 64, seed: int = 0, steps: int = 4000, lo: int = 64, hi: int = 1024):
    """n independent 2-D runs, sizes uniform in [lo, hi]^2, random walls, blobs, CFL 0.3."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n):
        ncells = (int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1)))
        bc = tuple(tuple("N" if rng.random() < 0.5 else "D" for _ in range(2)) for _ in range(2))
        out.append(Workload(f"plane_batch[{m}]", ncells, bc, 0.3, steps,
                            random_blobs(ncells, 4, 3.0, (0.5, 1.0), int(rng.integers(1 << 30)))))
    return out


def small(ncells, bc, cfl=0.3, steps=20, seed=0, nblobs=2, sigma_cells=2.0) -> Workload:
    """A small seeded case of any shape, for parity tests."""
    return Workload("small", tuple(ncells), tuple(tuple(b) for b in bc), cfl, steps,
                    random_blobs(ncells, nblobs, sigma_cells, (0.5, 1.0), seed)
                    if min(ncells) * DX > 8 * sigma_cells * DX else [])


def random_field(shape, seed: int) -> np.ndarray:
    """Standard-normal FP64 field (for per-step and transform parity cases)."""
    return np.random.default_rng(seed).standard_normal(shape)


def plane128_nn_dd(steps: int = 200) -> Workload:
    """The learned operator's box: 128 x 128 cells, Neumann walls on x,
    Dirichlet walls on y, CFL 0.3, half-step initial velocity, `steps` steps."""
    return Workload("plane128_nn_dd", (128, 128), (("N", "N"), ("D", "D")), 0.3, steps)


def sno_initial_pressures(n: int, seed: int, ncells=(128, 128), sigma_cells=(2.0, 8.0),
                          nblobs=(1, 6), amp_range=(-1.0, 1.0), dx=DX) -> np.ndarray:
    """n initial pressures on the full node lattice, shape (n, N0+1, N1+1), FP64.

    The learned operator's configured inputs: each sample is 1 to 6 Gaussian
    blobs (count uniform in `nblobs`), each with its own width sigma ~ U[2, 8]
    cells and amplitude ~ U[-1, 1], centred uniformly in [4 sigma, L - 4 sigma]
    per axis.  Generated with numpy's default_rng(seed).
    """
    rng = np.random.default_rng(seed)
    out = np.zeros((n,) + tuple(k + 1 for k in ncells))
    for s in range(n):
        nb = int(rng.integers(nblobs[0], nblobs[1] + 1))
        blobs = []
        for _ in range(nb):
            sig = float(rng.uniform(*sigma_cells)) * dx
            centre = tuple(float(rng.uniform(4 * sig, k * dx - 4 * sig)) for k in ncells)
            blobs.append(Blob(centre, sig, float(rng.uniform(*amp_range))))
        out[s] = Workload("sample", tuple(ncells), (), 0.3, 0, blobs, dx).p0_full()
    return out
