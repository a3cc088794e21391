"""Geometry descriptions of the workloads (plain data, no method arithmetic).

Shared by the oracle-side tests, the GPU-side tests and the benchmark.  The
ELT numbers follow the paper's parameter table and system-settings table
(Sec. 5.1): 39 m pupil with ~28 % central obstruction, 84x84 Shack-Hartmann
sensors, LGS at H = 90 km, alpha = 2, r0 = 0.129 m.  Where the paper gives no
value (layer profile, asterism of the benchmark, grid sizes) the workload
recipe below states the choice.
"""
import math
from dataclasses import dataclass, field
from typing import List

ARCSEC = math.pi / 648000.0


@dataclass
class GuideStar:
    theta_x: float  # direction [rad]
    theta_y: float
    H: float = 0.0  # LGS height [m]; 0 = natural guide star (no cone effect)
    n_sub: int = 0  # subapertures across its sensor; 0 = the geometry's n_sub


@dataclass
class Layer:
    h: float        # height [m]
    cn2: float      # fraction of the turbulence strength
    n: int          # layer grid size (n x n nodes, power of two)
    J: int          # wavelet levels
    delta: float = 1.0  # scaling constant delta_l of Eq. fewha


@dataclass
class Geometry:
    name: str
    D: float
    obstruction: float
    n_sub: int
    gs: List[GuideStar]
    layers: List[Layer]
    r0: float = 0.129
    L0: float = 25.0
    alpha: float = 2.0
    wavelet_N: int = 3   # Daubechies-3 (6 taps)
    k_recycle: int = 8
    snr: float = 10.0
    wind: List[tuple] = field(default_factory=list)  # per layer (speed m/s, direction rad)

    @property
    def n_unknowns(self):
        return sum(l.n * l.n for l in self.layers)

    def sensor_ns(self, g):
        """Subapertures across the sensor of guide star g."""
        return self.gs[g].n_sub or self.n_sub

    @property
    def n_slopes(self):
        return sum(2 * self.sensor_ns(g) ** 2 for g in range(len(self.gs)))


def _ring(n, radius_rad, H, phase=0.0):
    return [GuideStar(radius_rad * math.cos(phase + 2 * math.pi * k / n),
                      radius_rad * math.sin(phase + 2 * math.pi * k / n), H) for k in range(n)]


def _winds(n_layers, seed):
    import numpy as np
    rng = np.random.default_rng(seed)
    speeds = rng.uniform(5.0, 20.0, n_layers)
    dirs = rng.uniform(0.0, 2 * math.pi, n_layers)
    return [(float(s), float(d)) for s, d in zip(speeds, dirs)]


def tiny() -> Geometry:
    """8 m, 16x16 SH, 4 NGS at 30'' (azimuth 0/90/180/270 deg), layers 0 m / 8 km
    (Cn2 0.7 / 0.3) on 32x32 grids, Daubechies-3 with 3 levels."""
    return Geometry("tiny", D=8.0, obstruction=0.0, n_sub=16,
                    gs=_ring(4, 30 * ARCSEC, 0.0),
                    layers=[Layer(0.0, 0.7, 32, 3), Layer(8000.0, 0.3, 32, 3)],
                    r0=0.15, L0=25.0, wind=_winds(2, 1000))


def elt() -> Geometry:
    """39 m, 28 % obstruction, 6 LGS at 90 km on a 1' radius ring (60 deg
    steps), 84x84 SH; 9 layers at 0, 2, ..., 16 km with Cn2 ~ exp(-h/4 km),
    128x128 grids up to 8 km and 64x64 above; Daubechies-3 with 5 levels."""
    hs = [2000.0 * i for i in range(9)]
    w = [math.exp(-h / 4000.0) for h in hs]
    tot = sum(w)
    layers = [Layer(h, wi / tot, 128 if h <= 8000.0 else 64, 5) for h, wi in zip(hs, w)]
    return Geometry("elt", D=39.0, obstruction=0.28, n_sub=84,
                    gs=_ring(6, 60 * ARCSEC, 90000.0), layers=layers,
                    r0=0.129, L0=25.0, k_recycle=8, wind=_winds(9, 1001))


def ltao() -> Geometry:
    """The paper's LTAO asterism (Sec. 5.1): 3 NGS on a 10' diameter circle and
    6 LGS at 90 km on a 7.5' diameter circle, every sensor 80x80; 39 m pupil with
    28 % obstruction; the 9-layer profile of the ELT workload (128^2 up to 8 km,
    64^2 above; the wide NGS field makes the high layers' grids coarser)."""
    hs = [2000.0 * i for i in range(9)]
    w = [math.exp(-h / 4000.0) for h in hs]
    tot = sum(w)
    layers = [Layer(h, wi / tot, 128 if h <= 8000.0 else 64, 5) for h, wi in zip(hs, w)]
    return Geometry("ltao", D=39.0, obstruction=0.28, n_sub=80,
                    gs=_ring(3, 300 * ARCSEC, 0.0, phase=math.pi / 2) + _ring(6, 225 * ARCSEC, 90000.0),
                    layers=layers, r0=0.129, L0=25.0, k_recycle=8, wind=_winds(9, 1005))


def mcao() -> Geometry:
    """The paper's MCAO asterism (Sec. 5.1 and its system-settings table):
    6 LGS at 90 km with 84x84 sensors and 3 NGS with low-order sensors, one
    2x2 and two 1x1; the text puts the NGS on a 2 arcmin and the LGS on an
    8/3 arcmin diameter circle (the table swaps the two; the text is
    followed).  39 m pupil with 28 % obstruction; the 9-layer profile of the
    ELT workload."""
    hs = [2000.0 * i for i in range(9)]
    w = [math.exp(-h / 4000.0) for h in hs]
    tot = sum(w)
    layers = [Layer(h, wi / tot, 128 if h <= 8000.0 else 64, 5) for h, wi in zip(hs, w)]
    ngs = _ring(3, 60 * ARCSEC, 0.0, phase=math.pi / 2)
    for g, ns in zip(ngs, (2, 1, 1)):
        g.n_sub = ns
    return Geometry("mcao", D=39.0, obstruction=0.28, n_sub=84,
                    gs=ngs + _ring(6, 80 * ARCSEC, 90000.0), layers=layers,
                    r0=0.129, L0=25.0, k_recycle=8, wind=_winds(9, 1006))


def sizes() -> Geometry:
    """Small asterism with sensors of different sizes: LGS with 16x16 and
    12x12 sensors, NGS with 2x2 and 1x1 sensors, 3 layers (exercises the
    per-sensor paths of the operator at test size)."""
    gs = [GuideStar(20 * ARCSEC, 0.0, 90000.0), GuideStar(-10 * ARCSEC, 17 * ARCSEC, 90000.0, 12),
          GuideStar(-10 * ARCSEC, -17 * ARCSEC, 0.0, 2), GuideStar(30 * ARCSEC, 30 * ARCSEC, 0.0, 1)]
    return Geometry("sizes", D=8.0, obstruction=0.2, n_sub=16, gs=gs,
                    layers=[Layer(0.0, 0.5, 32, 3), Layer(4000.0, 0.3, 32, 3), Layer(9000.0, 0.2, 16, 2)],
                    r0=0.15, wind=_winds(3, 1007))


def medium() -> Geometry:
    """16 m, 40x40 SH, 4 LGS at 90 km on a 45'' ring, 5 layers on 64x64 grids
    (0-12 km), Daubechies-3 with 4 levels (the mid-size batched instance)."""
    hs = [0.0, 3000.0, 6000.0, 9000.0, 12000.0]
    w = [math.exp(-h / 4000.0) for h in hs]
    tot = sum(w)
    return Geometry("medium", D=16.0, obstruction=0.2, n_sub=40,
                    gs=_ring(4, 45 * ARCSEC, 90000.0, phase=math.pi / 4),
                    layers=[Layer(h, wi / tot, 64, 4) for h, wi in zip(hs, w)],
                    r0=0.15, wind=_winds(5, 1002))


def micro() -> Geometry:
    """2 m, 4x4 SH, one NGS and one LGS, two 8x8 layers with 2 wavelet levels:
    n = 128 unknowns, small enough for dense assembly and exact CG."""
    return Geometry("micro", D=2.0, obstruction=0.0, n_sub=4,
                    gs=[GuideStar(10 * ARCSEC, -5 * ARCSEC, 0.0),
                        GuideStar(-20 * ARCSEC, 15 * ARCSEC, 90000.0)],
                    layers=[Layer(0.0, 0.6, 8, 2), Layer(5000.0, 0.4, 8, 2, delta=1.5)],
                    r0=0.2, wind=_winds(2, 1003))


def mixed_ngs_lgs() -> Geometry:
    """Small mixed asterism: 2 NGS + 3 LGS, 3 layers of different sizes and
    scaling constants (exercises every code path of the operator)."""
    return Geometry("mixed", D=10.0, obstruction=0.25, n_sub=20,
                    gs=[GuideStar(40 * ARCSEC, 0.0, 0.0), GuideStar(-30 * ARCSEC, 25 * ARCSEC, 0.0)]
                    + _ring(3, 35 * ARCSEC, 90000.0, phase=0.3),
                    layers=[Layer(0.0, 0.5, 32, 3), Layer(4000.0, 0.3, 32, 4, delta=0.7),
                            Layer(10000.0, 0.2, 16, 2, delta=1.3)],
                    r0=0.14, wind=_winds(3, 1004))


CONFIGS = {"tiny": tiny, "elt": elt, "ltao": ltao, "mcao": mcao, "sizes": sizes, "medium": medium, "micro": micro,
           "mixed": mixed_ngs_lgs}


def get(name: str) -> Geometry:
    return CONFIGS[name]()
