"""Workload recipes: grid shapes, ensemble sizes, radii, tiles and input statistics.

A workload fixes everything needed to draw one synthetic assimilation problem:
the grid (longitudes x latitudes, levels, 3-D and 2-D variables), the
localisation radius r, the vertical reach, the number of members N, the
sub-domain tile, the ridge constant, and the statistics of the seeded fields
and of the observation network.  Components are labelled variable-major:
3-D variables first (each with `nlev` levels), then 2-D variables (one level);
within a level the order is latitude-major, longitude fastest.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Tuple


@dataclass(frozen=True)
class Workload:
    name: str
    nlon: int
    nlat: int
    nlev: int
    nvar_3d: int
    nvar_2d: int
    r: int
    N: int
    sub_lon: int
    sub_lat: int
    sigma2: Tuple[float, ...]          # background variance per variable
    corr_len: float = 3.0              # horizontal e-folding length, grid cells
    rho_vert: float = 0.5              # correlation between adjacent levels
    vert_reach: int = 1                # predecessors reach this many levels down
    lon_periodic: bool = True
    ridge_c: float = 1e-3              # lambda = ridge_c * tr(G) / p where p >= N - 1
    obs: str = "random"                # "random" or "every2"
    obs_frac: float = 0.5
    r_frac: float = 0.01               # R = r_frac * sigma2 of the observed variable
    seed: int = 1000

    @property
    def nvar(self) -> int:
        return self.nvar_3d + self.nvar_2d

    @property
    def n(self) -> int:
        return self.nlon * self.nlat * (self.nvar_3d * self.nlev + self.nvar_2d)

    def var_levels(self, v: int) -> int:
        return self.nlev if v < self.nvar_3d else 1

    def var_offset(self, v: int) -> int:
        off = 0
        for w in range(v):
            off += self.var_levels(w) * self.nlat * self.nlon
        return off

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# The five workloads of the study, plus small parity cases.
TINY_32x16 = Workload(  # one 2-D field, plain FP64 correctness case
    name="tiny_32x16_n20_r2", nlon=32, nlat=16, nlev=1, nvar_3d=1, nvar_2d=0,
    r=2, N=20, sub_lon=8, sub_lat=8, sigma2=(1.0,), corr_len=3.0,
    ridge_c=0.0, obs="every2", r_frac=0.01, seed=1000)

T63_N80 = Workload(  # SPEEDY-T63-shaped state, 7 levels x {u, v, T, q} + ps
    name="t63_192x96x29_n80_r2", nlon=192, nlat=96, nlev=7, nvar_3d=4, nvar_2d=1,
    r=2, N=80, sub_lon=12, sub_lat=12, sigma2=(25.0, 25.0, 4.0, 1e-6, 1e4),
    corr_len=4.0, rho_vert=0.5, obs="random", obs_frac=0.5, r_frac=0.01, seed=2000)

T63_N40 = T63_N80.with_(name="t63_192x96x29_n40_r2", N=40, seed=4000)

T127_N96 = Workload(  # T127-shaped scale case
    name="t127_384x192x29_n96_r3", nlon=384, nlat=192, nlev=7, nvar_3d=4, nvar_2d=1,
    r=3, N=96, sub_lon=12, sub_lat=12, sigma2=(1.0, 1.0, 1.0, 1.0, 1.0),
    corr_len=3.0, rho_vert=0.5, obs="random", obs_frac=0.3, r_frac=0.01, seed=5000)

# Parity cases small enough for the oracle: several tiles, a ragged tile
# edge in both directions, the longitude seam, the poles, two variable kinds.
SMALL_3D = Workload(
    name="small_40x30x2x2+1_n48_r2", nlon=40, nlat=30, nlev=2, nvar_3d=2, nvar_2d=1,
    r=2, N=48, sub_lon=12, sub_lat=12, sigma2=(4.0, 1e-2, 1e3),
    corr_len=3.0, rho_vert=0.5, obs="random", obs_frac=0.5, r_frac=0.01, seed=7000)

# Same grid with N = 24: p >= N - 1 on most rows (ridge), D spans nine orders of
# magnitude and the sub-domain blocks reach condition numbers near 1e11.
SMALL_ILL = SMALL_3D.with_(name="small_40x30x2x2+1_n24_r2_ill", N=24)

SMALL_R1 = Workload(
    name="small_28x20x3x1_n32_r1", nlon=28, nlat=20, nlev=3, nvar_3d=1, nvar_2d=0,
    r=1, N=32, sub_lon=8, sub_lat=6, sigma2=(1.0,), corr_len=2.0,
    obs="random", obs_frac=0.3, seed=7100)

# Same grid with N = 16: p > N / 2 on most rows (the rows a single-precision
# problem regresses in double precision); p <= 14 < N - 1, so no ridge.
SMALL_R1_N16 = SMALL_R1.with_(name="small_28x20x3x1_n16_r1", N=16, seed=7110)

# Ridge active: p >= N - 1 for most rows (r = 3 with N = 24).
SMALL_RIDGE = Workload(
    name="small_36x24x2x1_n24_r3_ridge", nlon=36, nlat=24, nlev=2, nvar_3d=1, nvar_2d=0,
    r=3, N=24, sub_lon=12, sub_lat=12, sigma2=(2.0,), corr_len=3.0,
    obs="random", obs_frac=0.5, ridge_c=1e-3, seed=7200)

# T63 statistics (N = 80, r = 2, no ridge) on a grid the oracle finishes in seconds.
SMALL_T63 = Workload(
    name="small_48x26x3x1+1_n80_r2", nlon=48, nlat=26, nlev=3, nvar_3d=1, nvar_2d=1,
    r=2, N=80, sub_lon=12, sub_lat=12, sigma2=(25.0, 1e4), corr_len=4.0, rho_vert=0.5,
    obs="random", obs_frac=0.5, r_frac=0.01, seed=7300)

# Same statistics with N = 120: four members per lane on 30 lanes in the
# register regressions.
SMALL_T63_N120 = SMALL_T63.with_(name="small_48x26x3x1+1_n120_r2", N=120, seed=7310)

# Two 2-D fields, r = 3: 27 predecessor slots (one level, ring longitude).
SMALL_2D_R3 = Workload(
    name="small_40x30x0+2_n64_r3", nlon=40, nlat=30, nlev=1, nvar_3d=0, nvar_2d=2,
    r=3, N=64, sub_lon=12, sub_lat=12, sigma2=(1.0, 1e2), corr_len=3.0,
    obs="random", obs_frac=0.5, r_frac=0.01, seed=7400)

# Accuracy study (radius and tile size against the analysis RMSE of Eq. 18 over
# filter cycles): a 96 x 48 grid, 3 levels of two 3-D variables and one 2-D
# variable, N = 60 (at N = 40, r = 2 puts rows at p = N - 2, below the ridge
# threshold with one residual degree of freedom); the study varies r and the tile.
STUDY = Workload(
    name="study_96x48x3x2+1_n60", nlon=96, nlat=48, nlev=3, nvar_3d=2, nvar_2d=1,
    r=2, N=60, sub_lon=12, sub_lat=12, sigma2=(4.0, 1.0, 1e2), corr_len=4.0, rho_vert=0.5,
    obs="random", obs_frac=0.5, r_frac=0.01, seed=7500)

WORKLOADS = {w.name: w for w in (TINY_32x16, T63_N80, T63_N40, T127_N96, STUDY,
                                 SMALL_3D, SMALL_ILL, SMALL_R1, SMALL_R1_N16, SMALL_RIDGE,
                                 SMALL_T63, SMALL_T63_N120, SMALL_2D_R3)}


def batch_instances(count: int = 256, base_seed: int = 3000):
    """The batch of independent problems of uneven size: instance i (seed
    base_seed + i) draws its grid from 24 x 12 to 96 x 48 (nlon in {24, 36, ...,
    96}, nlat = nlon / 2), 1-7 levels, 1-5 variables, N in [20, 120] and
    r in {1, 2, 3, 4}; fields as in the 32 x 16 case (correlation length 3 cells,
    unit variance, vertical correlation 0.5), half of the components observed
    with R = 0.01, 12 x 12 sub-domains (ragged at the edges)."""
    from .philox import uint32_stream
    out = []
    for i in range(count):
        seed = base_seed + i
        k = [int(x) for x in uint32_stream(seed, 9, 6)]
        nlon = 24 + 12 * (k[0] % 7)
        nlev = 1 + k[1] % 7
        nvar = 1 + k[2] % 5
        N = 20 + k[3] % 101
        r = 1 + k[4] % 4
        out.append(Workload(
            name=f"batch{i:03d}_{nlon}x{nlon // 2}x{nlev}x{nvar}_n{N}_r{r}", nlon=nlon,
            nlat=nlon // 2, nlev=nlev, nvar_3d=nvar, nvar_2d=0, r=r, N=N, sub_lon=12,
            sub_lat=12, sigma2=(1.0,) * nvar, corr_len=3.0, rho_vert=0.5, obs="random",
            obs_frac=0.5, r_frac=0.01, ridge_c=1e-3, seed=seed))
    return out
