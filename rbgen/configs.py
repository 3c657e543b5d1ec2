"""Acquisition configurations (ring, grid, fan and frequency schedule).

Three workloads, named for what they are:

* ``tiny``      — 64-element ring of radius 50 mm, 64x64 grid at 1.6 mm,
                  64 rays per emitter, 0.3/0.4/0.5 MHz as three sets of one.
* ``breast256`` — 256-element ring of radius 110 mm, 256x256 grid at 0.9 mm,
                  256 rays per emitter, 12 frequencies 0.3-1.0 MHz in 4 sets of 3.
* ``breast512`` — same ring, 512x512 grid at 0.45 mm, 256 rays per emitter,
                  20 frequencies 0.3-1.25 MHz in 5 sets of 4.
* ``invivo512`` — 512 elements on the same ring (the in-vivo transducer count),
                  256x256 grid at 0.9 mm, 512 rays per emitter, 5 sets of 4.
* ``fullring1024`` — the same with all 1024 elements of the array.
* ``ring`` / ``batch_mix`` / ``poisson_requests`` — workloads of uneven sizes on the
                  same 110 mm ring (batched reconstructions and a request stream).

The ring of 256 elements with an 11 cm radius, the 1480 m/s water speed and
the low-to-high sweep over sets of consecutive frequencies are the paper's
in-vitro acquisition (Sec. 4.1); the grid pitches and frequency counts are
synthetic workload choices.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple


@dataclasses.dataclass(frozen=True)
class Config:
    name: str
    n_elem: int            # ring elements; each is emitter and receiver
    ring_radius: float     # [m]
    nx: int
    ny: int
    h: float               # pixel pitch [m]
    n_rays: int            # rays per emitter fan
    freqs_hz: Tuple[float, ...]
    sets: Tuple[Tuple[int, ...], ...]   # indices into freqs_hz, low -> high
    power_y: float         # absorption power-law exponent
    c_water: float = 1480.0
    seed: int = 20251116
    kind: str = "ellipses"  # phantom family: "ellipses" or "breast"

    @property
    def npix(self) -> int:
        return self.nx * self.ny

    @property
    def ds(self) -> float:
        """Ray step: half a pixel."""
        return self.h / 2.0

    @property
    def max_steps(self) -> int:
        return int(math.ceil(4.0 * self.ring_radius / self.ds))

    @property
    def support_margin(self) -> float:
        return max(2e-3, 2.0 * self.h)

    def set_freqs(self, j: int) -> List[float]:
        return [self.freqs_hz[i] for i in self.sets[j]]


def _sets(n: int, per: int) -> Tuple[Tuple[int, ...], ...]:
    return tuple(tuple(range(k, k + per)) for k in range(0, n, per))


def _linspace_hz(lo_mhz: float, hi_mhz: float, n: int) -> Tuple[float, ...]:
    if n == 1:
        return (lo_mhz * 1e6,)
    return tuple((lo_mhz + (hi_mhz - lo_mhz) * k / (n - 1)) * 1e6 for k in range(n))


def tiny(**kw) -> Config:
    base = dict(name="tiny", n_elem=64, ring_radius=0.050, nx=64, ny=64, h=1.6e-3, n_rays=64,
                freqs_hz=(0.3e6, 0.4e6, 0.5e6), sets=((0,), (1,), (2,)), power_y=1.0,
                seed=20251116 + 0, kind="ellipses")
    base.update(kw)
    return Config(**base)


def breast256(**kw) -> Config:
    f = _linspace_hz(0.3, 1.0, 12)
    base = dict(name="breast256", n_elem=256, ring_radius=0.110, nx=256, ny=256, h=0.9e-3, n_rays=256,
                freqs_hz=f, sets=_sets(12, 3), power_y=1.1, seed=20251116 + 1, kind="breast")
    base.update(kw)
    return Config(**base)


def breast512(**kw) -> Config:
    f = _linspace_hz(0.3, 1.25, 20)
    base = dict(name="breast512", n_elem=256, ring_radius=0.110, nx=512, ny=512, h=0.45e-3, n_rays=256,
                freqs_hz=f, sets=_sets(20, 4), power_y=1.1, seed=20251116 + 2, kind="breast")
    base.update(kw)
    return Config(**base)


def invivo512(**kw) -> Config:
    """The paper's in-vivo acquisition size (Sec. 4.2: 512 transducers, images on a ~1 mm
    grid): 512 elements on the 110 mm ring, 256 x 256 pixels at 0.9 mm, 512 rays per
    emitter, 20 frequencies 0.3-1.25 MHz in 5 sets of 4."""
    base = dict(name="invivo512", n_elem=512, n_rays=512, seed=20251116 + 6)
    base.update(kw)
    return ring(512, 256, 20, **{k: v for k, v in base.items() if k not in ("n_elem",)})


def fullring1024(**kw) -> Config:
    """The full 1024-element array the in-vivo data come from (Sec. 4.2 uses half of it):
    1024 elements on the 110 mm ring, 256 x 256 pixels at 0.9 mm, 512 rays per emitter,
    5 sets of 4 frequencies 0.3-1.25 MHz."""
    base = dict(name="fullring1024", n_rays=512, seed=20251116 + 7)
    base.update(kw)
    return ring(1024, 256, 20, **base)


CONFIGS = {"tiny": tiny, "breast256": breast256, "breast512": breast512, "invivo512": invivo512,
           "fullring1024": fullring1024}


def config_by_name(name: str, **kw) -> Config:
    return CONFIGS[name](**kw)


def ring(n_elem: int, n_grid: int, n_freq: int, per_set: int = 4, f_lo_mhz: float = 0.3, f_hi_mhz: float = 1.25,
         n_rays: int = 256, seed: int = 20251116 + 3, name: str = "ring", **kw) -> Config:
    """A breast-phantom workload on the 110 mm ring with n_elem elements and an n_grid^2
    grid whose half-width is 5 % beyond the ring; n_freq frequencies in sets of per_set."""
    R = 0.110
    h = 2.0 * 1.05 * R / (n_grid - 1)
    f = _linspace_hz(f_lo_mhz, f_hi_mhz, n_freq)
    base = dict(name=name, n_elem=n_elem, ring_radius=R, nx=n_grid, ny=n_grid, h=h, n_rays=n_rays, freqs_hz=f,
                sets=_sets(n_freq, per_set), power_y=1.1, seed=seed, kind="breast")
    base.update(kw)
    return Config(**base)


def batch_mix(n: int = 16, rings=(128, 256, 512), grids=(256, 512, 768), freqs=(8, 24), seed: int = 20251116 + 4,
              **kw) -> List[Config]:
    """n reconstructions of uneven sizes: ring sizes and grid sizes drawn from the given
    lists, frequency counts uniform in [freqs[0], freqs[1]] rounded to whole sets of 4."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        ne = int(rng.choice(rings))
        ng = int(rng.choice(grids))
        nf = int(rng.integers(freqs[0] // 4, freqs[1] // 4 + 1)) * 4
        out.append(ring(ne, ng, nf, seed=seed + 1 + k, name=f"mix{k}_{ne}el_{ng}px_{nf}f", **kw))
    return out


def poisson_requests(rate_hz: float, count: int, rings=(128, 256, 512), grids=(256, 512, 768, 1024), sets=(3, 6),
                     per_set: int = 4, seed: int = 20251116 + 5, **kw) -> List[Tuple[float, Config]]:
    """count requests with exponential inter-arrival times of mean 1 / rate_hz seconds;
    ring and grid sizes drawn from the lists, 3-6 frequency sets of per_set."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(count):
        t += float(rng.exponential(1.0 / rate_hz))
        ne = int(rng.choice(rings))
        ng = int(rng.choice(grids))
        ns = int(rng.integers(sets[0], sets[1] + 1))
        out.append((t, ring(ne, ng, ns * per_set, per_set=per_set, seed=seed + 1 + k,
                            name=f"req{k}_{ne}el_{ng}px_{ns}sets", **kw)))
    return out
