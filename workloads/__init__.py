"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module only draws sample matrices X (T samples x N variables, float64,
row-major).  It holds none of the estimator's arithmetic: no ranking, no
copula transform, no covariance estimate, no entropy.  Both the FP64 CPU
oracle and the CUDA path consume exactly the arrays produced here.

Workload recipes (all draws from numpy.random.Generator(PCG64(seed))):

* ``random_corr(rng, N)``: W ~ N(0,1)^{NxN}, A = W W^T + 0.5 I,
  Sigma = D^{-1/2} A D^{-1/2} with D = diag(A) (a random correlation matrix).
* ``plain``: X = xi @ chol(Sigma)^T, xi ~ N(0,1)^{TxN}.  Sizes of the small
  exhaustive case: N=10, T=500, seed 0 (968 nplets of orders 3..10).
* ``ar1``: N independent AR(1) series e_t = phi e_{t-1} + sqrt(1-phi^2) xi_t
  with e_0 ~ N(0,1) (stationary, unit variance), mixed as x_t = chol(Sigma) e_t.
  fMRI-shaped stand-in: N=20, T=1200, phi=0.7, seed 1.  The paper's fMRI
  recordings (anesthesia study) are not available; this series stands in.
* ``planted``: N=30, T=1000, seed 2.  Variables 0-9 share a latent
  z ~ N(0,1): x_i = z + 0.5 xi_i (redundancy).  Variables 10-18 are iid
  N(0,1) and variable 19 = -(x_10 + ... + x_18) + 0.3 xi (synergy).
  Variables 20-29 iid N(0,1).  Stands in for the paper's N=30 iid benchmark
  system (its timing does not depend on the distribution).
* ``multi``: 64 datasets; dataset d uses seed 3000+d, draws N ~ U{10..40} and
  T ~ U{200..2000} first, then X as in ``plain``.  Stands in for the paper's
  collection of 920 heterogeneous datasets (not available here).
* ``plain`` with N=60, T=2000, seed 4: the differentiation workload.
* ``paired``: P subjects x 2 conditions (datasets 0..P-1 condition A,
  P..2P-1 condition B; subject p in both).  Subject p draws (seed 5000+p) a
  random correlation R_p; the network matrix B has 11 blocks of 5 variables
  (1 on the diagonal, 0.6 inside a block, 0 elsewhere); condition c mixes
  Sigma_pc = (1 - w_c) R_p + w_c B with w_A = 0.5, w_B = 0.3 (weaker
  within-network coupling in B).  X is N AR(1) series (phi = 0.7, as in
  ``ar1``) mixed by chol(Sigma_pc), condition A drawn before B.  Stands in
  for the anesthesia study (16 subjects, awake and deep, 55 regions in 11
  networks of 5); the recordings are not available and their length is not
  stated, T = 300 is assumed.
"""
from __future__ import annotations

import numpy as np

SEEDS = {"small": 0, "ar1": 1, "planted": 2, "multi_base": 3000, "grad": 4,
         "paired_base": 5000}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_corr(rng: np.random.Generator, N: int) -> np.ndarray:
    """Random correlation matrix D^{-1/2}(W W^T + 0.5 I)D^{-1/2}."""
    W = rng.standard_normal((N, N))
    A = W @ W.T + 0.5 * np.eye(N)
    d = np.sqrt(np.diag(A))
    return A / np.outer(d, d)


def plain(N: int, T: int, seed: int) -> np.ndarray:
    """T x N Gaussian samples with a random correlation matrix."""
    rng = _rng(seed)
    S = random_corr(rng, N)
    L = np.linalg.cholesky(S)
    xi = rng.standard_normal((T, N))
    return np.ascontiguousarray(xi @ L.T)


def ar1(N: int = 20, T: int = 1200, seed: int = 1, phi: float = 0.7) -> np.ndarray:
    """N AR(1) series (stationary start) mixed by chol of a random correlation."""
    rng = _rng(seed)
    S = random_corr(rng, N)
    L = np.linalg.cholesky(S)
    e = np.empty((T, N))
    e[0] = rng.standard_normal(N)
    s = np.sqrt(1.0 - phi * phi)
    xi = rng.standard_normal((T - 1, N))
    for t in range(1, T):
        e[t] = phi * e[t - 1] + s * xi[t - 1]
    return np.ascontiguousarray(e @ L.T)


def planted(T: int = 1000, seed: int = 2) -> np.ndarray:
    """30 variables: redundant block 0-9, synergistic block 10-19, iid 20-29."""
    rng = _rng(seed)
    N = 30
    X = np.empty((T, N))
    z = rng.standard_normal(T)
    X[:, 0:10] = z[:, None] + 0.5 * rng.standard_normal((T, 10))
    X[:, 10:19] = rng.standard_normal((T, 9))
    X[:, 19] = -X[:, 10:19].sum(axis=1) + 0.3 * rng.standard_normal(T)
    X[:, 20:30] = rng.standard_normal((T, 10))
    return X


def multi(D: int = 64, base_seed: int = 3000):
    """List of D (X, N, T) with per-dataset N ~ U{10..40}, T ~ U{200..2000}."""
    out = []
    for d in range(D):
        rng = _rng(base_seed + d)
        N = int(rng.integers(10, 41))
        T = int(rng.integers(200, 2001))
        S = random_corr(rng, N)
        L = np.linalg.cholesky(S)
        xi = rng.standard_normal((T, N))
        out.append(np.ascontiguousarray(xi @ L.T))
    return out


def _ar1_mix(rng: np.random.Generator, S: np.ndarray, T: int, phi: float) -> np.ndarray:
    N = S.shape[0]
    L = np.linalg.cholesky(S)
    e = np.empty((T, N))
    e[0] = rng.standard_normal(N)
    s = np.sqrt(1.0 - phi * phi)
    xi = rng.standard_normal((T - 1, N))
    for t in range(1, T):
        e[t] = phi * e[t - 1] + s * xi[t - 1]
    return np.ascontiguousarray(e @ L.T)


def paired(P: int = 16, N: int = 55, T: int = 300, base_seed: int = 5000,
           block: int = 5, w=(0.5, 0.3), phi: float = 0.7):
    """2P datasets: subjects 0..P-1 in condition A, then the same subjects in
    condition B (dataset p pairs with dataset P + p)."""
    B = np.zeros((N, N))
    for b0 in range(0, N, block):
        B[b0:b0 + block, b0:b0 + block] = 0.6
    np.fill_diagonal(B, 1.0)
    A_sets, B_sets = [], []
    for p in range(P):
        rng = _rng(base_seed + p)
        R = random_corr(rng, N)
        A_sets.append(_ar1_mix(rng, (1 - w[0]) * R + w[0] * B, T, phi))
        B_sets.append(_ar1_mix(rng, (1 - w[1]) * R + w[1] * B, T, phi))
    return A_sets + B_sets


# Named workloads: (X, orders).  Orders are inclusive ranges of subset sizes.
def small():
    return plain(10, 500, SEEDS["small"]), list(range(3, 11))


def fmri_like():
    return ar1(20, 1200, SEEDS["ar1"]), list(range(3, 21))


def planted30():
    return planted(1000, SEEDS["planted"]), list(range(3, 31))


def grad60():
    return plain(60, 2000, SEEDS["grad"]), [3, 4, 5]


def multi64():
    Xs = multi(64, SEEDS["multi_base"])
    return Xs, [list(range(3, min(X.shape[1], 8) + 1)) for X in Xs]


def paired55():
    """16 subjects x 2 conditions, N = 55, orders 3..6 (exhaustive)."""
    return paired(16, 55, 300, SEEDS["paired_base"]), [3, 4, 5, 6]
