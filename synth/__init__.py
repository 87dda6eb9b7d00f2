"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

Holds none of the method's arithmetic: only random numbers and the parameters
of the synthetic workloads.  Both the GPU path's callers and the CPU oracle
draw their inputs from here, so the two sides see identical inputs.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) -> 53-bit uniforms in [0, 1) -> Box-Muller
(1958) for N(0, 1).  Seed of right-hand side `rhs` of problem `problem` in
workload `config`: 1000 config + 16 problem + rhs.
"""
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, count):
    """count consecutive SplitMix64 outputs (uint64) from state `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, count):
    """53-bit uniforms in [0, 1)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed, count):
    """N(0,1) samples by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:count]


def rhs_seed(config, problem, rhs):
    return 1000 * config + 16 * problem + rhs


def normal_rhs(N, nrhs, config, problem=0, first=0):
    """Column-major (N, nrhs) float64 block of seeded N(0,1) right-hand sides."""
    B = np.empty((N, nrhs), dtype=np.float64, order="F")
    for j in range(nrhs):
        B[:, j] = normal(rhs_seed(config, problem, first + j), N)
    return B


def batched_problems(count=64, seed=3000, n_lo=6, n_hi=16, k_lo=1.0, k_hi=10.0):
    """Batched workload: `count` problems with mesh n ~ U{n_lo..n_hi} and
    kappa ~ U[k_lo, k_hi] drawn from SplitMix64(seed)."""
    u = uniform(seed, 2 * count)
    out = []
    for p in range(count):
        n = n_lo + min(int(u[2 * p] * (n_hi - n_lo + 1)), n_hi - n_lo)
        kappa = k_lo + (k_hi - k_lo) * u[2 * p + 1]
        out.append((n, float(kappa)))
    return out


def serving_requests(count=200, seed=5000, n_lo=8, n_hi=32, k_lo=1.0, k_hi=12.0,
                     r_lo=1, r_hi=16, rate=1.0):
    """Serving workload: Poisson arrivals (exponential gaps with mean 1/rate
    seconds), n ~ U{n_lo..n_hi}, kappa ~ U[k_lo, k_hi], nrhs ~ U{r_lo..r_hi}."""
    u = uniform(seed, 4 * count)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log(1.0 - u[4 * i]) / rate
        n = n_lo + min(int(u[4 * i + 1] * (n_hi - n_lo + 1)), n_hi - n_lo)
        kappa = k_lo + (k_hi - k_lo) * u[4 * i + 2]
        nrhs = r_lo + min(int(u[4 * i + 3] * (r_hi - r_lo + 1)), r_hi - r_lo)
        out.append({"id": i, "t": t, "n": n, "kappa": float(kappa), "nrhs": nrhs})
    return out


def perturbed_kuhn_mesh(n, amplitude, seed):
    """A non-lattice tetrahedral mesh of the unit cube (input recipe): the n^3
    sub-cubes cut into 6 tetrahedra along the axis permutations, vertex id
    (i (n+1) + j)(n+1) + k, and every vertex off the cube's faces moved by
    amplitude / n times a seeded uniform draw in [-1, 1)^3.  amplitude < 0.25
    inverts no tetrahedron.  Returns (coords float64
    [(n+1)^3, 3], tets int32 [6 n^3, 4])."""
    idx = np.arange(n + 1)
    I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")
    lat = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)
    vid = lambda p: (p[..., 0] * (n + 1) + p[..., 1]) * (n + 1) + p[..., 2]
    c = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), axis=-1).reshape(-1, 3)
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        p = c.copy()
        corners = [vid(p)]
        for ax in perm:
            p = p.copy()
            p[:, ax] += 1
            corners.append(vid(p))
        tets.append(np.stack(corners, axis=1))
    # tet of sub-cube ci and permutation pi at row 6 ci + pi
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    coords = lat.astype(np.float64) / n
    inner = np.all((lat > 0) & (lat < n), axis=1)
    u = uniform(seed, 3 * len(coords)).reshape(-1, 3)
    coords = coords + np.where(inner[:, None], (2.0 * u - 1.0) * amplitude / n, 0.0)
    return coords, tets
