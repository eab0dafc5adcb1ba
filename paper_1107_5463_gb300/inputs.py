"""Seeded synthetic inputs shared by the tests and the bench.

This module holds no arithmetic of the Metropolis method: it only draws
configurations, couplings and parameter ladders with numpy's seeded generator,
shaped like the workloads of Weigel & Yavors'kii (Section 2 and Table 1):
periodic square and simple-cubic lattices, +-1 Ising spins, angles and unit
vectors for continuous spins, bimodal +-J couplings for the Edwards-Anderson
spin glass.  Both the CUDA path and the CPU oracle consume what it returns.
"""
import math

import numpy as np

DEFAULT_SEED = 0x5EED20111107546

# critical couplings used by the workloads
BETA_C_2D_ISING = 0.5 * math.log(1.0 + math.sqrt(2.0))      # ln(1+sqrt2)/2
BETA_3D_ISING = 0.2216546
BETA_3D_HEISENBERG = 0.693
BETAS_2D_XY = (0.9, 1.12, 1.4)
EA_SIZES = (8, 12, 16, 24, 32)


def rng(seed):
    return np.random.default_rng(seed)


def nsites(d, L):
    return L ** d


def ising_spins(d, L, seed):
    """Uniform random +-1 int8 configuration in natural order."""
    return np.where(rng(seed).random(nsites(d, L)) < 0.5, -1, 1).astype(np.int8)


def ising_bonds(d, L, seed, p_zero=0.0):
    """Forward-bond couplings (d, N) in {-1, +1} (or 0 with probability p_zero)."""
    g = rng(seed)
    jb = np.where(g.random((d, nsites(d, L))) < 0.5, -1, 1).astype(np.int8)
    if p_zero > 0:
        jb[g.random(jb.shape) < p_zero] = 0
    return jb


def float_bonds(d, L, seed):
    """Forward-bond couplings (d, N) drawn uniformly from [-1, 1]."""
    return rng(seed).uniform(-1.0, 1.0, (d, nsites(d, L))).astype(np.float32)


def angles(d, L, seed):
    """Uniform angles in [0, 2 pi), FP64."""
    return rng(seed).uniform(0.0, 2.0 * math.pi, nsites(d, L))


def unit_vectors(d, L, seed):
    """Unit vectors uniform on the sphere, (N, 3) FP64."""
    v = rng(seed).normal(size=(nsites(d, L), 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def two_spin_bonds(d, L, site_a, mu):
    """All couplings zero except the forward bond of site_a along mu."""
    jb = np.zeros((d, nsites(d, L)), np.int8)
    jb[mu, site_a] = 1
    return jb


def ea_sample_sizes(nsamples, sizes=EA_SIZES):
    """Side of each disorder sample: sizes[s mod len(sizes)]."""
    return [sizes[s % len(sizes)] for s in range(nsamples)]


def geometric_betas(ntemps, beta_min=0.5, beta_max=3.0):
    """ntemps inverse temperatures spaced geometrically in [beta_min, beta_max]."""
    if ntemps == 1:
        return np.array([beta_min])
    k = np.arange(ntemps)
    return beta_min * (beta_max / beta_min) ** (k / (ntemps - 1))
