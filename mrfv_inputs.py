"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the method (no equation of state, no flux, no
prediction): it only draws the parameters of the initial data from a seed and names
the workloads.  Both sides receive the same parameter vectors and sample the initial
data themselves.

Random numbers come from splitmix64 (S. Vigna's published 64-bit mixer; the state is
advanced by the golden-ratio increment and the output mixed by two xor-shift-multiply
rounds), mapped to doubles in [0, 1) from the top 53 bits.

Initial-data kinds (the integer codes are part of the C interface and of the oracle):

* ``IC_QUADRANTS`` (2D): four constant states, one per quadrant of the domain, in the
  order of the paper's Table 1 (I top-right, II top-left, III bottom-left,
  IV bottom-right).  16 parameters: (rho, v1, v2, p) for I, II, III, IV.
* ``IC_ELLIPSOID`` (3D): axis-aligned ellipsoid at rest; 10 parameters
  (cx, cy, cz, a, b, c, rho_in, p_in, rho_out, p_out); inside means
  ((x-cx)/a)^2 + ((y-cy)/b)^2 + ((z-cz)/c)^2 < 1.
* ``IC_SHOCKTUBE`` (2D/3D): planar Riemann problem normal to one axis; 8 parameters
  (axis, x0, rho_L, u_L, p_L, rho_R, u_R, p_R); left means x_axis < x0, u is the
  velocity along the axis.
* ``IC_UNIFORM``: constant state, 5 parameters (rho, v1, v2, v3, p).
* ``IC_WAVE``: smooth periodic density wave advected by a constant velocity,
  5 parameters (amp, v1, v2, v3, p); rho = 1 + amp*sin(2*pi*(x1+x2[+x3])).
* ``IC_ROTATED_ELLIPSOID`` (3D, the paper's Section 4.2 case): 10 parameters
  (a, b, c, r_c, theta, phi, rho_in, rhoe_in, rho_out, rhoe_out), fluid at rest.
"""
from __future__ import annotations

import math

IC_QUADRANTS = 0
IC_ELLIPSOID = 1
IC_SHOCKTUBE = 2
IC_UNIFORM = 3
IC_WAVE = 4
IC_ROTATED_ELLIPSOID = 5

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream (Vigna); ``next_double`` maps the top 53 bits to [0, 1)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def next_double(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.next_double()


def quadrant_params(seed: int) -> list[float]:
    """Four seeded quadrant states: rho in [0.5, 2], v1, v2 in [-0.75, 0.75], p in [0.3, 1.5]."""
    g = SplitMix64(seed)
    out: list[float] = []
    for _ in range(4):
        rho = g.uniform(0.5, 2.0)
        v1 = g.uniform(-0.75, 0.75)
        v2 = g.uniform(-0.75, 0.75)
        p = g.uniform(0.3, 1.5)
        out += [rho, v1, v2, p]
    return out


def laxliu6_params() -> list[float]:
    """Lax-Liu configuration 6, the paper's Table 1 (quadrants I, II, III, IV)."""
    return [1.00, 0.75, -0.50, 1.00,
            2.00, 0.75, 0.50, 1.00,
            1.00, -0.75, 0.50, 1.00,
            3.00, -0.75, -0.50, 1.00]


def ellipsoid_params(seed: int, rho_out: float = 1.0) -> list[float]:
    """Axis-aligned blast ellipsoid at the origin: semi-axes U[0.2, 0.4];
    inside rho=1, p=10; outside p=0.1 and rho=rho_out.  The default is the
    workload's alternative rho_out=1: with rho_out=0.1 the AUSM+ step at rest
    drives the outer cells to negative pressure at CFL >= 0.3."""
    g = SplitMix64(seed)
    a = g.uniform(0.2, 0.4)
    b = g.uniform(0.2, 0.4)
    c = g.uniform(0.2, 0.4)
    return [0.0, 0.0, 0.0, a, b, c, 1.0, 10.0, rho_out, 0.1]


def paper3d_params() -> list[float]:
    """The paper's rotated ellipsoid (Section 4.2): a=1/3, b=1, c=3, r_c=3/5,
    theta=pi/3, phi=pi/4; rho 0.125 / 1 and rho*e 0.25 / 2.5 inside / outside."""
    return [1.0 / 3.0, 1.0, 3.0, 3.0 / 5.0, math.pi / 3.0, math.pi / 4.0,
            0.125, 0.25, 1.0, 2.5]


def sod_params(axis: int = 0, x0: float = 0.5) -> list[float]:
    """Sod's shock tube along ``axis``: (1, 0, 1) | (0.125, 0, 0.1)."""
    return [float(axis), x0, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1]


# Workloads named by what they are (sizes follow the paper's 2D and 3D Riemann set-ups).
WORKLOADS = {
    "uniform2d_fp64_128": dict(dim=2, precision="fp64", levels=4, base_blocks=(2, 2, 1),
                               lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), adapt=False,
                               cfl=0.5, steps=200, eps=1e-3, ic=IC_QUADRANTS),
    "mr2d_fp32_L7": dict(dim=2, precision="fp32", levels=8, base_blocks=(1, 1, 1),
                         lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), adapt=True,
                         cfl=0.5, eps=1e-3, t_end=0.25, ic=IC_QUADRANTS),
    "amr2d_lts_fp32": dict(dim=2, precision="fp32", levels=4, base_blocks=(16, 16, 1),
                           lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), adapt=True, lts=True,
                           criterion="grad", eps_w=0.05, eta_tol=0.8,
                           cfl=0.5, ic=IC_QUADRANTS),
    "mr3d_blast_fp32_L4": dict(dim=3, precision="fp32", levels=5, base_blocks=(2, 2, 2),
                               lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), adapt=True,
                               cfl=0.5, eps=1e-3, ic=IC_ELLIPSOID),
}
