"""Unpreconditioned GMRES (Saad and Schultz), as used for Eq. (3.2) in Section 3.8.

TEST INFRASTRUCTURE: part of the CPU oracle.

Steps, in the textbook order:
  r0 = b - A x0, beta = |r0|, v1 = r0 / beta;
  for k = 1, 2, ...: w = A v_k; modified Gram-Schmidt against v_1..v_k gives the
  Hessenberg column h_{1..k,k}; h_{k+1,k} = |w|, v_{k+1} = w / h_{k+1,k};
  earlier Givens rotations are applied to the new column, a new rotation zeroes
  h_{k+1,k}, and the rotated right-hand side g gives the residual estimate |g_{k+1}|;
  stop when |g_{k+1}| / |b| <= tol (or at maxit, or at the restart length);
  solve the k x k upper-triangular system for y and set x = x0 + V y.
The stopping test is on the relative residual |b - A x| / |b|, as in Matlab's gmres. The
true residual is recomputed at the end (one more product), so a solve of n iterations
uses n + 2 products when it converges in its first cycle, matching the paper's count.
"""
from __future__ import annotations

import math

import numpy as np


def gmres(matvec, b, x0, tol: float = 1e-10, maxit: int = 100, restart=None):
    """Return (x, iterations, true relative residual, number of matvec calls)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    m = int(restart) if restart else int(maxit)
    bnorm = float(np.linalg.norm(b))
    nmv = 0
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, nmv
    iters = 0
    while True:
        r = b - matvec(x)
        nmv += 1
        beta = float(np.linalg.norm(r))
        if beta / bnorm <= tol or iters >= maxit:
            return x, iters, beta / bnorm, nmv
        V = [r / beta]
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        k_used = 0
        for k in range(m):
            w = matvec(V[k])
            nmv += 1
            # modified Gram-Schmidt
            for j in range(k + 1):
                H[j, k] = float(np.dot(w, V[j]))
                w = w - H[j, k] * V[j]
            hk1 = float(np.linalg.norm(w))
            H[k + 1, k] = hk1
            # previous rotations on the new column
            for j in range(k):
                t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            # new rotation that zeroes H[k+1, k]
            d = math.hypot(H[k, k], H[k + 1, k])
            if d == 0.0:
                cs[k], sn[k] = 1.0, 0.0
            else:
                cs[k], sn[k] = H[k, k] / d, H[k + 1, k] / d
            H[k, k] = d
            H[k + 1, k] = 0.0
            gvec[k + 1] = -sn[k] * gvec[k]
            gvec[k] = cs[k] * gvec[k]
            iters += 1
            k_used = k + 1
            done = abs(gvec[k + 1]) / bnorm <= tol or iters >= maxit or hk1 == 0.0
            if not done and k + 1 < m:
                V.append(w / hk1)
            if done:
                break
        # back substitution on the k_used x k_used upper-triangular system
        y = np.zeros(k_used)
        for i in range(k_used - 1, -1, -1):
            y[i] = (gvec[i] - np.dot(H[i, i + 1:k_used], y[i + 1:k_used])) / H[i, i]
        for i in range(k_used):
            x = x + y[i] * V[i]
        if abs(gvec[k_used]) / bnorm <= tol or iters >= maxit:
            r = b - matvec(x)
            nmv += 1
            return x, iters, float(np.linalg.norm(r)) / bnorm, nmv
