"""Seeded synthetic workload descriptions shared by the oracle, the tests and the bench.

This module holds *inputs only*: grid sizes, domains, coefficient parameters,
initial-datum parameters, seeds and path counts.  It contains none of the
method's arithmetic (no operators, no Brownian functionals, no Magnus terms),
so both the CPU oracle and the CUDA path may import it without sharing any
computation.

The Brownian paths themselves are not stored anywhere: each side regenerates
them from (seed, global path index, fine index) with its own implementation of
the Philox4x32-10 counter-based generator (Salmon et al., SC'11).

Workload shapes follow the paper's experiments (Section 3: Langevin SPDE on a
square (x, v) box, zero Dirichlet boundary, Gaussian initial datum, T = 1,
Lebesgue grid 1e-4) and the five benchmark configurations of this project.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import Tuple

COEF_CONST = 0
COEF_TRIG = 1

# x profile psi of the variable-coefficient operators (Eq. coeffsLangevinVar):
# g^vv(x) = a psi(x), sigma^v(x) = sigma sqrt(psi(x)).
XPROF_NONE = 0        # psi = 1: the constant-coefficient operators
XPROF_RATIONAL = 1    # psi(x) = 1 + c / (1 + x^2); c = 1 is the paper's choice


@dataclass(frozen=True)
class Workload:
    """One seeded synthetic problem.

    d            interior grid points per axis (n_x = n_v = d, Eq. xGrid/vGrid)
    ax, bx       x-domain, Delta x = (bx - ax) / (d + 1)
    av, bv       v-domain
    drift_sign   kappa in f^x(x, v) = kappa * v  (the SPDE is written with +v d_x,
                 the paper's experiments use -v, Eq. coeffsLangevinConst)
    kind         COEF_CONST: a(t) = a0, sigma(t) = s0
                 COEF_TRIG:  a(t) = a0 + a1 sin(2 pi t), sigma(t) = s0 (1 + s1 cos(2 pi t))
    u0_mean      mean (x, v) of the Gaussian initial datum
    u0_cov       covariance (xx, xv, vv) of the Gaussian initial datum
    u0_scale     multiplier c0 of the normalised Gaussian density (1 = density,
                 2 pi = the paper's unnormalised exp(-(x^2+v^2)/2))
    T            terminal time
    n_fine       number of fine Brownian increments on [0, T] (Lebesgue grid)
    paths        number of Brownian paths
    seed         64-bit Philox key
    path_offset  global index of the first path (paths are keyed by global index)
    x_profile    XPROF_NONE or XPROF_RATIONAL (x-dependent g^vv and sigma^v)
    x_profile_c  the constant c of the rational profile
    """

    name: str
    d: int
    ax: float
    bx: float
    av: float
    bv: float
    drift_sign: int = 1
    kind: int = COEF_CONST
    a0: float = 1.0
    a1: float = 0.0
    s0: float = 0.5
    s1: float = 0.0
    u0_mean: Tuple[float, float] = (0.0, 0.0)
    u0_cov: Tuple[float, float, float] = (1.0, 0.0, 1.0)
    u0_scale: float = 1.0
    T: float = 1.0
    n_fine: int = 10_000
    paths: int = 100
    seed: int = 20220719
    path_offset: int = 0
    x_profile: int = XPROF_NONE
    x_profile_c: float = 1.0

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# Small Langevin case: d = 32 on [-5, 5]^2, +v d_x drift, a = 1, sigma = 0.5,
# standard Gaussian density, 100 paths, Lebesgue grid 1e-4 over [0, 1].
LANGEVIN_32 = Workload(
    name="langevin_const_d32", d=32, ax=-5.0, bx=5.0, av=-5.0, bv=5.0,
    drift_sign=1, kind=COEF_CONST, a0=1.0, s0=0.5,
    u0_mean=(0.0, 0.0), u0_cov=(1.0, 0.0, 1.0), u0_scale=1.0,
    T=1.0, n_fine=10_000, paths=100, seed=20220719)

# Time-dependent coefficients: d = 128 on [-6, 6]^2, a(t) = 1 + 0.5 sin(2 pi t),
# sigma(t) = 0.5 (1 + 0.3 cos(2 pi t)), u0 = N((0.5, 0), diag(0.5, 1)),
# 4096 paths, 2^14 fine increments on [0, 1].
LANGEVIN_TRIG_128 = Workload(
    name="langevin_trig_d128", d=128, ax=-6.0, bx=6.0, av=-6.0, bv=6.0,
    drift_sign=1, kind=COEF_TRIG, a0=1.0, a1=0.5, s0=0.5, s1=0.3,
    u0_mean=(0.5, 0.0), u0_cov=(0.5, 0.0, 1.0), u0_scale=1.0,
    T=1.0, n_fine=16_384, paths=4096, seed=20220720)

# Uneven batch: grids 64^2, 128^2, 256^2 in ratio 4:2:1 of 16384 paths,
# constant a = 1, sigma = 0.5 on [-6, 6]^2, standard Gaussian.
BATCH_GRIDS = tuple(
    Workload(name=f"langevin_const_d{d}", d=d, ax=-6.0, bx=6.0, av=-6.0, bv=6.0,
             drift_sign=1, kind=COEF_CONST, a0=1.0, s0=0.5,
             T=1.0, n_fine=16_384, paths=p, seed=20220721 + i)
    for i, (d, p) in enumerate(((64, 9362), (128, 4681), (256, 2341))))

# Large grid: d = 512 on [-8, 8]^2, a = 1, sigma in {0.25, 0.5, 1.0}, 1024 paths.
LARGE_512 = tuple(
    Workload(name=f"langevin_const_d512_s{s}", d=512, ax=-8.0, bx=8.0, av=-8.0, bv=8.0,
             drift_sign=1, kind=COEF_CONST, a0=1.0, s0=s,
             T=1.0, n_fine=16_384, paths=1024, seed=20220722)
    for s in (0.25, 0.5, 1.0))

# The paper's own constant-coefficient setting (Section 3.1): -v d_x drift,
# a = 1.1, sigma = 1/sqrt(10), phi = exp(-(x^2+v^2)/2), domain [-4, 4]^2.
PAPER_CONST = Workload(
    name="paper_langevin_const", d=100, ax=-4.0, bx=4.0, av=-4.0, bv=4.0,
    drift_sign=-1, kind=COEF_CONST, a0=1.1, s0=10.0 ** -0.5,
    u0_scale=2.0 * 3.141592653589793, T=1.0, n_fine=10_000, paths=100, seed=2207)


# The paper's variable-coefficient setting (Section 3.2, Table errorsVar): the
# constant case above with g^vv = a (1 + 1/(x^2+1)), sigma^v = sigma sqrt(1 + 1/(x^2+1)),
# d = 100, 200, 300; the reference is Euler-Maruyama with step 1e-5, so the fine
# Brownian grid has 10^5 cells on [0, 1].
PAPER_VAR = tuple(
    Workload(name=f"paper_langevin_var_d{d}", d=d, ax=-4.0, bx=4.0, av=-4.0, bv=4.0,
             drift_sign=-1, kind=COEF_CONST, a0=1.1, s0=10.0 ** -0.5,
             u0_scale=2.0 * 3.141592653589793, T=1.0, n_fine=100_000, paths=100, seed=2208,
             x_profile=XPROF_RATIONAL, x_profile_c=1.0)
    for d in (100, 200, 300))


def path_range(paths: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous [start, stop) block of global path indices owned by `rank`."""
    base, rem = divmod(paths, world)
    start = rank * base + min(rank, rem)
    return start, start + base + (1 if rank < rem else 0)
