"""Dense FP64 routes to the psi-score for small N (TEST INFRASTRUCTURE ONLY).

Three independent formulations, each a plain transcription of the paper:

* ``direct_psi``: the N per-origin systems at once, P = (I - A)^{-1} B (Eq. 11),
  Q = C P + D (Eq. 7 in matrix form), psi^T = 1^T Q / N (Eq. 9).  With N right-hand
  sides this is the "N wall systems" computation the method replaces.
* ``one_system_psi``: the paper's single system, s solves (I - A)^T s = c (the limit of
  Eq. 13), psi^T = (s^T B + d^T) / N (Eq. 12).
* ``balance_psi``: for every origin i, the scalar balance equations of the walls
  (Eqs. 2-3) and newsfeeds (Eqs. 4-5) solved as one 2N x 2N system in the unknowns
  p_i^(n), q_i^(n), then psi_i by Eq. 1.  This route never forms A, B, C or D, so it
  checks their definitions.

Reading: a user with no leaders has an empty newsfeed; its balance equation (Eq. 4)
degenerates to 0 = 0 and is replaced by p^(n) = 0 (its row of A and B is zero).
numpy.linalg.solve (LAPACK LU with partial pivoting) is the only library step.
"""
from __future__ import annotations

import numpy as np


def leader_sets(n, follower, leader):
    """L(j) for every j, as sets (duplicates merged).  Self-loops are not allowed."""
    sets = [set() for _ in range(n)]
    for j, i in zip(np.asarray(follower).tolist(), np.asarray(leader).tolist()):
        if j == i:
            raise ValueError("self-loop")
        sets[j].add(i)
    return sets


def matrices(n, follower, leader, lam, mu):
    """A, B, c, d entry by entry from the definitions after Eqs. 6-7."""
    lam = np.asarray(lam, np.float64)
    mu = np.asarray(mu, np.float64)
    L = leader_sets(n, follower, leader)
    A = np.zeros((n, n))
    B = np.zeros((n, n))
    for j in range(n):
        sig = sum(lam[k] + mu[k] for k in sorted(L[j]))
        for i in L[j]:
            A[j, i] = mu[i] / sig
            B[j, i] = lam[i] / sig
    c = mu / (lam + mu)
    d = lam / (lam + mu)
    return A, B, c, d


def direct_psi(n, follower, leader, lam, mu):
    A, B, c, d = matrices(n, follower, leader, lam, mu)
    P = np.linalg.solve(np.eye(n) - A, B)          # Eq. 11
    Q = np.diag(c) @ P + np.diag(d)                # Eq. 7
    return np.ones(n) @ Q / n                      # Eq. 9


def one_system_psi(n, follower, leader, lam, mu, return_s=False):
    A, B, c, d = matrices(n, follower, leader, lam, mu)
    s = np.linalg.solve((np.eye(n) - A).T, c)      # s^T (I - A) = c^T
    psi = (s @ B + d) / n                          # Eq. 12
    return (psi, s) if return_s else psi


def balance_psi(n, follower, leader, lam, mu):
    lam = np.asarray(lam, np.float64)
    mu = np.asarray(mu, np.float64)
    L = leader_sets(n, follower, leader)
    psi = np.zeros(n)
    for i in range(n):
        # unknowns x = [p^(0..n-1), q^(0..n-1)] for posts of origin i
        M = np.zeros((2 * n, 2 * n))
        r = np.zeros(2 * n)
        for j in range(n):
            if L[j]:
                # Eqs. 4-5: sum_{k in L(j)} (lam_k + mu_k) p^(j) = lam_i 1{i in L(j)} + sum_{k in L(j)} mu_k p^(k)
                M[j, j] += sum(lam[k] + mu[k] for k in L[j])
                for k in L[j]:
                    M[j, k] -= mu[k]
                r[j] = lam[i] if i in L[j] else 0.0
            else:
                M[j, j] = 1.0  # empty newsfeed: p^(j) = 0
            # Eqs. 2-3: (lam_j + mu_j) q^(j) = mu_j p^(j) + lam_i 1{j = i}
            M[n + j, n + j] = lam[j] + mu[j]
            M[n + j, j] = -mu[j]
            r[n + j] = lam[i] if j == i else 0.0
        x = np.linalg.solve(M, r)
        psi[i] = x[n:].sum() / n                   # Eq. 1
    return psi


def pagerank_dense(n, follower, leader, alpha, weights=None):
    """Solution of pi^T (I - alpha W) = (1-alpha)/N 1^T (fixed point of Eq. 22).

    W_ji = w_i / sum_{l in L(j)} w_l for i in L(j) (w = 1: W = D_out^{-1} L); rows of users
    without leaders are zero (no dangling redistribution)."""
    L = leader_sets(n, follower, leader)
    w = np.ones(n) if weights is None else np.asarray(weights, np.float64)
    W = np.zeros((n, n))
    for j in range(n):
        tot = sum(w[k] for k in L[j])
        for i in L[j]:
            W[j, i] = w[i] / tot
    return np.linalg.solve((np.eye(n) - alpha * W).T, np.full(n, (1 - alpha) / n))
