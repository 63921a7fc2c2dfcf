"""Seeded synthetic problem definitions for the GIS hot path.

This module is the one piece the CUDA path and the CPU oracle both use: it
holds problem *definitions* (dynamics name and parameters, constraint box X,
root grid, sample lattice, sampled control values, levels) and a SplitMix64
generator (Steele, Lea & Flood 2014, "Fast splittable pseudorandom number
generators") for the randomised batches. It contains none of the method's
arithmetic.

The paper runs no public benchmark or dataset; its only workload is the
dimensional CSTR of Sec. 4.1 (Eq. 4, Table 2). The five workloads below are
synthetic systems with the shapes the method is exercised on: 2-D and 4-D
state boxes, uniform root grids, inclusive sample lattices, a finite set of
control values, and 0-3 levels of boundary-only subdivision (Sec. 3.1).
"""
from __future__ import annotations

import math

MASK64 = (1 << 64) - 1
SEED_BASE = 0x6153


class SplitMix64:
    """SplitMix64 as published (golden-gamma increment, two xor-shift-multiply rounds)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        return a + (b - a) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, a: int, b: int) -> int:
        """Uniform integer in [a, b]."""
        return a + self.next_u64() % (b - a + 1)

    def log_uniform(self, a: float, b: float) -> float:
        return math.exp(self.uniform(math.log(a), math.log(b)))

    def exponential(self, mean: float) -> float:
        return -mean * math.log(1.0 - self.uniform())


def controls_grid(lo: float, hi: float, count: int) -> list[list[float]]:
    """`count` evenly spaced scalar control values from lo to hi, inclusive."""
    if count == 1:
        return [[0.5 * (lo + hi)]]
    return [[lo + i * (hi - lo) / (count - 1)] for i in range(count)]


# ---------------------------------------------------------------- dynamics ----
def vdp(mu: float = 1.0) -> dict:
    return {"dyn": "vdp", "n": 2, "m": 1, "params": [mu]}


def cstr_dl(Da: float = 0.072, B: float = 8.0, beta: float = 0.3, gamma: float = 20.0) -> dict:
    return {"dyn": "cstr_dl", "n": 2, "m": 1, "params": [Da, B, beta, gamma]}


def cartpole(mc: float = 1.0, mp: float = 0.1, l: float = 0.5, g: float = 9.81) -> dict:
    return {"dyn": "cartpole", "n": 4, "m": 1, "params": [mc, mp, l, g]}


# Table 2 of the paper: q, V, c_Af, T_f, E/R, k0, -dH, UA, c_p, rho
CSTR_PAPER_PARAMS = [100.0, 100.0, 1.0, 350.0, 8750.0, 7.2e10, 5.0e4, 5.0e4, 0.239, 1000.0]


def cstr_paper() -> dict:
    return {"dyn": "cstr_paper", "n": 2, "m": 1, "params": list(CSTR_PAPER_PARAMS)}


def linmap(A, B) -> dict:
    n = len(A)
    m = len(B[0])
    flat = [float(v) for row in A for v in row] + [float(v) for row in B for v in row]
    return {"dyn": "linmap", "n": n, "m": m, "params": flat}


def problem(dyn: dict, lo, hi, n0, k, controls, dt, substeps, levels=0, rule="inner",
            precision="fp32", band=None, name="") -> dict:
    n = dyn["n"]
    if isinstance(n0, int):
        n0 = [n0] * n
    p = dict(dyn)
    p.update({"lo": [float(v) for v in lo], "hi": [float(v) for v in hi], "n0": list(n0), "k": k,
              "controls": [[float(v) for v in c] for c in controls], "dt": float(dt),
              "substeps": substeps, "levels": levels, "rule": rule, "precision": precision,
              "name": name})
    if band is not None:
        p["band"] = band
    return p


# ------------------------------------------------------------ the workloads ----
def vdp_64(levels: int = 0, n0: int = 64, precision: str = "fp64") -> dict:
    """Controlled Van der Pol mu = 1, X = [-3,3]^2, 64^2 cells, 3x3 samples,
    u in {-1,-0.5,0,0.5,1}, dt = 0.1 by 10 RK4 substeps, no subdivision, FP64."""
    return problem(vdp(1.0), [-3, -3], [3, 3], n0, 3, controls_grid(-1, 1, 5), 0.1, 10,
                   levels=levels, precision=precision, name=f"vdp_{n0}")


def cstr_256(levels: int = 3, n0: int = 256, precision: str = "fp32") -> dict:
    """Dimensionless CSTR Da = 0.072, X = [0,1] x [0,8], 256^2 root cells, 4x4
    samples, 11 controls in [-2,2], dt = 0.05 by 4 RK4 substeps, 3 levels of
    2x2 boundary subdivision, FP32 with FP64 recheck."""
    return problem(cstr_dl(0.072), [0, 0], [1, 8], n0, 4, controls_grid(-2, 2, 11), 0.05, 4,
                   levels=levels, precision=precision, name=f"cstr_{n0}_L{levels}")


def cartpole_48(levels: int = 2, n0: int = 48, precision: str = "fp32") -> dict:
    """Cart-pole (m_c 1, m_p 0.1, l 0.5, g 9.81), X = [-2.4,2.4] x [-3,3] x
    [-0.4,0.4] x [-3,3], 48^4 cells, 2^4 corner samples, 9 forces in [-10,10],
    dt = 0.02 by one RK4 step, 2 subdivision levels, FP32 with FP64 recheck."""
    return problem(cartpole(), [-2.4, -3, -0.4, -3], [2.4, 3, 0.4, 3], n0, 2,
                   controls_grid(-10, 10, 9), 0.02, 1, levels=levels, precision=precision,
                   name=f"cartpole_{n0}_L{levels}")


def cstr_paper_problem(n0=(16, 16), levels: int = 0, n_u: int = 7, substeps: int = 10) -> dict:
    """The paper's own CSTR (Eq. 4, Table 2): X = [0,1] x [345,355],
    U = [285,315], sampling period h = 0.1 min (RK4, `substeps` substeps)."""
    return problem(cstr_paper(), [0.0, 345.0], [1.0, 355.0], list(n0), 3,
                   controls_grid(285.0, 315.0, n_u), 0.1, substeps, levels=levels,
                   name="cstr_paper")


def _random_2d(rng: SplitMix64, lo_cells: float, hi_cells: float, precision: str) -> dict:
    kind = "vdp" if rng.uniform() < 0.5 else "cstr"
    count = rng.log_uniform(lo_cells, hi_cells)
    n0 = max(2, int(round(math.sqrt(count))))
    n_u = rng.randint(5, 11)
    levels = rng.randint(0, 3)
    if kind == "vdp":
        mu = rng.uniform(0.5, 2.0)
        return problem(vdp(mu), [-3, -3], [3, 3], n0, 3, controls_grid(-1, 1, n_u), 0.1, 10,
                       levels=levels, precision=precision, name=f"vdp_mu{mu:.3f}_{n0}")
    Da = rng.uniform(0.06, 0.09)
    return problem(cstr_dl(Da), [0, 0], [1, 8], n0, 3, controls_grid(-2, 2, n_u), 0.05, 4,
                   levels=levels, precision=precision, name=f"cstr_Da{Da:.4f}_{n0}")


def batch_512(count: int = 512, seed: int = SEED_BASE + 3, max_cells: float = 512.0 ** 2) -> list[dict]:
    """512 uneven instances, 50/50 Van der Pol (mu ~ U[0.5,2]) / CSTR
    (Da ~ U[0.06,0.09]); cells log-uniform in [32^2, 512^2] (n0 = round(sqrt));
    3x3 samples; 5-11 controls; 0-3 levels; FP32 with FP64 recheck."""
    rng = SplitMix64(seed)
    return [_random_2d(rng, 32.0 ** 2, max_cells, "fp32") for _ in range(count)]


def serving_2000(count: int = 2000, seed: int = SEED_BASE + 5, mean_gap_s: float = 0.005,
                 max_2d_cells: float = 1024.0 ** 2, max_4d_n0: float = 48.0) -> list[dict]:
    """Poisson-arrival requests (mean 200/s), one third each Van der Pol, CSTR
    and cart-pole; 2-D grids log-uniform 32^2..1024^2 cells, 4-D n0
    log-uniform in [16, 48]; 0-3 levels. Each dict carries `arrival_s`."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(mean_gap_s)
        kind = rng.randint(0, 2)
        if kind < 2:
            p = _random_2d(rng, 32.0 ** 2, max_2d_cells, "fp32")
        else:
            n0 = int(round(rng.log_uniform(16.0, max_4d_n0)))
            p = cartpole_48(levels=rng.randint(0, 3), n0=n0)
        p["arrival_s"] = t
        p["request_id"] = i
        out.append(p)
    return out


WORKLOADS = {
    "vdp_64": vdp_64,
    "cstr_256": cstr_256,
    "cartpole_48": cartpole_48,
}
