"""Named synthetic workloads (sizes and seeds only; no arithmetic of the method).

The paper's own runs (Sec. 3) are periodic L x L Ising lattices with J = 1,
random initial spins, 80% flatness and ln f halved down to a final value; it
uses no dataset.  These entries fix the sizes and seeds of the workloads this
library is tested and measured on.  Seeds follow 20150811 + 1000 * id +
replicate.
"""
from __future__ import annotations

from dataclasses import dataclass, replace


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    n_win_E: int
    n_win_M: int
    overlap_E: float
    overlap_M: float
    walkers_per_window: int
    lnf_init: float
    lnf_final: float
    lnf_factor: float
    flatness: float
    exchange_interval: int      # trials per walker per cycle
    check_every: int            # cycles between flatness checks
    ident: int

    def seed(self, replicate: int = 0) -> int:
        return 20150811 + 1000 * self.ident + replicate

    @property
    def N(self) -> int:
        return self.L * self.L

    @property
    def n_walkers(self) -> int:
        return self.n_win_E * self.n_win_M * self.walkers_per_window

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


# Plain serial 2D WL: L=4, one window over all (E, M), one walker.
SERIAL_L4 = Workload("serial_wl_L4", 4, 1, 1, 0.75, 0.75, 1, 1.0, 1e-6, 0.5, 0.8, 10_000, 1, 1)
# 2D REWL: L=8, 3x3 windows at 75% overlap, 4 walkers per window, exchange every 1e4 trials.
REWL_L8 = Workload("rewl_L8_3x3_w4", 8, 3, 3, 0.75, 0.75, 4, 1.0, 1e-6, 0.5, 0.8, 10_000, 1, 2)
# Batched 2D REWL: L=32, 16x4 windows at 75% overlap, 32 walkers per window (2048 walkers).
REWL_L32 = Workload("rewl_L32_16x4_w32", 32, 16, 4, 0.75, 0.75, 32, 1.0, 1e-6, 0.5, 0.8, 10_000, 8, 3)
# Precision study: L=64, 32x8 windows at 75% overlap, 16 walkers per window, ln f down to 1e-8.
REWL_L64 = Workload("rewl_L64_32x8_w16", 64, 32, 8, 0.75, 0.75, 16, 1.0, 1e-8, 0.5, 0.8, 10_000, 16, 4)

# The paper's own runs (Sec. 3): E split into 3 equal windows at 50% overlap,
# M unrestricted, 3 walkers per window, ln f down to 1e-8; L = 8 and 16.
PAPER_L8 = Workload("paper_L8_E3_o50_w3", 8, 3, 1, 0.5, 0.5, 3, 1.0, 1e-8, 0.5, 0.8, 10_000, 1, 6)
PAPER_L16 = Workload("paper_L16_E3_o50_w3", 16, 3, 1, 0.5, 0.5, 3, 1.0, 1e-8, 0.5, 0.8, 10_000, 1, 7)
# Serial 2D WL over the whole (E, M) range at L = 8, one walker (the
# reference of the Eq. 5 comparison in Sec. 3).
SERIAL_L8 = Workload("serial_wl_L8", 8, 1, 1, 0.5, 0.5, 1, 1.0, 1e-8, 0.5, 0.8, 10_000, 1, 8)

# Uneven batch: 24 independent REWL runs, six each of L = 16, 24, 32, 48 with
# window grids and walkers per window scaled to L (4x2/32, 8x2/16, 12x4/16,
# 16x4/8; 10,752 walkers in all), 75% overlap, ln f down to 1e-6.
BATCH_SPECS = ((16, 4, 2, 32), (24, 8, 2, 16), (32, 12, 4, 16), (48, 16, 4, 8))


def mixed_batch() -> list:
    out = []
    for L, nE, nM, W in BATCH_SPECS:
        for r in range(6):
            out.append(Workload(f"batch_L{L}_{nE}x{nM}_w{W}_r{r}", L, nE, nM, 0.75, 0.75, W, 1.0, 1e-6, 0.5, 0.8,
                                10_000, 8, 5))
    return out


BATCH_NAME = "batch_24_mixed_L16_24_32_48"

ALL = {w.name: w for w in (SERIAL_L4, REWL_L8, REWL_L32, REWL_L64, PAPER_L8, PAPER_L16, SERIAL_L8)}
