"""Seeded synthetic inputs shared by the CUDA path, its tests and the oracle.

This module holds no arithmetic of the method: only random draws.  Everything
the method computes from them (the Taylor-Green field, He scaling of initial
weights, ...) is done independently on each side.
"""
import numpy as np

# Seed of the Taylor-Green perturbation (the arXiv number of the paper).
TGV_SEED = 0x220711571
TGV_EPS = 1e-6


def perturbation(shape, seed=TGV_SEED, eps=TGV_EPS):
    """Uniform draws in [-eps, eps), float64, PCG64 stream of ``seed``."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-eps, eps, size=shape)


def random_conserved(shape, seed, rho=(1.0, 0.2), mom=0.5, rhoE=(178.6, 5.0)):
    """A random (non-smooth) state in conserved variables, shape (5, *shape):
    rho ~ rho[0] + rho[1] U(-1,1), rho v_i ~ mom U(-1,1), rho e ~ rhoE[0] + rhoE[1] U(-1,1)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, size=(5,) + tuple(shape))
    q = np.empty_like(u)
    q[0] = rho[0] + rho[1] * u[0]
    q[1:4] = mom * u[1:4]
    q[4] = rhoE[0] + rhoE[1] * u[4]
    return q


def uniform_draws(dims, seed):
    """One U(-1, 1) array of shape (dims[l+1], dims[l]) per dense layer (initial weights)."""
    rng = np.random.default_rng(seed)
    return [rng.uniform(-1.0, 1.0, size=(dims[l + 1], dims[l])) for l in range(len(dims) - 1)]


def normal(shape, seed, scale=1.0):
    """Standard normal draws times ``scale``."""
    return scale * np.random.default_rng(seed).standard_normal(size=shape)


def epoch_permutation(n, seed, epoch):
    """Shuffle order of ``n`` training samples for one epoch."""
    return np.random.default_rng([seed, epoch]).permutation(n).astype(np.int64)


def batch_members(n=12, seed=12, Re=(30.0, 200.0, 1600.0), K=(8, 12, 16), P=(3, 6)):
    """n independent (K, P, Re) draws for a batch of Taylor-Green instances of uneven size."""
    rng = np.random.default_rng(seed)
    return [(int(rng.choice(K)), int(rng.choice(P)), float(rng.choice(Re))) for _ in range(n)]
