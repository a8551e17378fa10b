"""Seeded synthetic inputs for the domain-wall solver workloads.

This module only draws random numbers and packs them into arrays.  It holds
none of the operator's arithmetic, so both the CPU oracle and the CUDA path
(tests, bench, smoke) take their inputs from here without sharing method code.

Layouts (canonical, complex, x0 fastest):
  * gauge links, U(1):  U[mu][x_{nd-1}]...[x_0]           (complex scalar)
  * gauge links, SU(3): U[mu][x_{nd-1}]...[x_0][a][b]     (3x3 complex)
  * 5-d spinor:         psi[s][x_{nd-1}]...[x_0][spin][color]

The paper's Monte Carlo Schwinger-model ensembles (Sec. 3) are not available;
link angles drawn i.i.d. from N(0, sigma) stand in for them.  Their mean
plaquette is exp(-2 sigma^2), so sigma = 0.5 is a rough field (about
beta = 1.5 in the paper's units) and sigma = 0.214 is close to beta = 6.
"""
from __future__ import annotations

import dataclasses
import numpy as np


def volume(dims) -> int:
    v = 1
    for L in dims:
        v *= int(L)
    return v


def rng_for(seed: int) -> np.random.Generator:
    """numpy PCG64 generator; every workload draws the gauge field first."""
    return np.random.default_rng(int(seed))


def u1_angles(rng: np.random.Generator, dims, sigma: float) -> np.ndarray:
    """Link angles theta_mu(x) ~ N(0, sigma), shape (nd, V), float64."""
    return rng.normal(0.0, float(sigma), size=(len(dims), volume(dims)))


def u1_links(theta: np.ndarray) -> np.ndarray:
    """U_mu(x) = exp(i theta_mu(x)), complex128, same shape as theta."""
    return np.exp(1j * theta)


def gaussian_complex(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex Gaussian array: real and imaginary parts each N(0, 1)."""
    z = rng.standard_normal(tuple(shape) + (2,))
    return z[..., 0] + 1j * z[..., 1]


def spinor_shape(dims, Ls: int, group: str):
    nspin = 2 if len(dims) == 2 else 4
    ncol = 1 if group == "u1" else 3
    return (int(Ls), volume(dims), nspin, ncol)


def gaussian_spinor(rng: np.random.Generator, dims, Ls: int, group: str = "u1") -> np.ndarray:
    """Gaussian 5-d source, canonical layout flattened to shape (Ls, V, nspin, ncol)."""
    return gaussian_complex(rng, spinor_shape(dims, Ls, group))


def su3_links(rng: np.random.Generator, dims, eps: float = 0.3) -> np.ndarray:
    """U = exp(i eps H), H the traceless Hermitian part of a complex Gaussian 3x3.

    The exponential is taken through H's eigen-decomposition and the result is
    re-unitarised by its polar factor.  Shape (nd, V, 3, 3), complex128.
    """
    nd = len(dims)
    V = volume(dims)
    G = gaussian_complex(rng, (nd, V, 3, 3))
    H = 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[..., None, None] * np.eye(3)
    w, Q = np.linalg.eigh(H)
    U = (Q * np.exp(1j * eps * w)[..., None, :]) @ np.conj(np.swapaxes(Q, -1, -2))
    W, _, Vh = np.linalg.svd(U)
    return W @ Vh


def gauge_transform_u1(rng: np.random.Generator, V: int) -> np.ndarray:
    """Random U(1) gauge rotation g(x) = exp(i phi(x)), phi uniform in [0, 2 pi)."""
    return np.exp(1j * rng.uniform(0.0, 2.0 * np.pi, size=V))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic lattice problem: geometry, parameters and seed."""
    name: str
    dims: tuple
    Ls: int
    group: str          # "u1" or "su3"
    sigma: float        # U(1) angle width; SU(3): the exponent scale eps
    M5: float           # domain-wall height (positive convention)
    mf: float
    seed: int

    @property
    def nd(self) -> int:
        return len(self.dims)

    @property
    def V(self) -> int:
        return volume(self.dims)

    def links(self):
        """Return (links, rng) with the gauge field drawn first from the seed."""
        rng = rng_for(self.seed)
        if self.group == "u1":
            theta = u1_angles(rng, self.dims, self.sigma)
            return u1_links(theta), rng
        return su3_links(rng, self.dims, self.sigma), rng

    def angles(self):
        """U(1) only: (theta, rng), theta the link angles drawn first."""
        assert self.group == "u1"
        rng = rng_for(self.seed)
        return u1_angles(rng, self.dims, self.sigma), rng

    def draw(self, nsrc: int = 1):
        """(U, [sources...]) drawn in order gauge field, then sources."""
        U, rng = self.links()
        srcs = [gaussian_spinor(rng, self.dims, self.Ls, self.group) for _ in range(nsrc)]
        return U, srcs


# Workload shapes of the 2-d Schwinger-model study (Sec. 3) and their 4-d and
# batched extensions.  Coordinates are (L0, L1, ...), x0 fastest.
SCHWINGER_32 = Workload("u1_2d_32x32_Ls8", (32, 32), 8, "u1", 0.5, 1.0, 0.01, 1001)
SCHWINGER_256 = Workload("u1_2d_256x256_Ls16", (256, 256), 16, "u1", 0.7, 1.0, 0.005, 1002)
SCHWINGER_256_SMOOTH = Workload("u1_2d_256x256_Ls16_smooth", (256, 256), 16, "u1", 0.214, 1.0, 0.005, 1002)
SCHWINGER_128_GRAD = Workload("u1_2d_128x128_Ls12", (128, 128), 12, "u1", 0.7, 1.0, 0.005, 1004)
SCHWINGER_1024 = Workload("u1_2d_1024x1024_Ls16", (1024, 1024), 16, "u1", 0.7, 1.0, 0.005, 1006)
SU3_16x32 = Workload("su3_4d_16x16x16x32_Ls16", (16, 16, 16, 32), 16, "su3", 0.3, 1.8, 0.01, 1005)
# the coarse-Ls study of the paper's discussion (a 128^2 field near beta 6, outer Ls = 32)
SCHWINGER_128_LS32 = Workload("u1_2d_128x128_Ls32_smooth", (128, 128), 32, "u1", 0.214, 1.0, 0.01, 1007)


def batched_classes():
    """Mixed-size multi-RHS batch: 64 sources, sizes (64, 128, 256)[i mod 3].

    One gauge field per size class (seed 1003 + class), shared by that class.
    Returns a list of (Workload, n_sources).
    """
    out = []
    for c, L in enumerate((64, 128, 256)):
        n = len([i for i in range(64) if i % 3 == c])
        out.append((Workload(f"u1_2d_{L}x{L}_Ls16_batch", (L, L), 16, "u1", 0.7, 1.0, 0.005, 1003 + c), n))
    return out
