"""An independent, tiny numpy lattice Boltzmann step, written for cross-checking.

It shares nothing with the oracle: its velocity set is enumerated in a
different order, its weights are solved from the lattice isotropy conditions,
the equilibrium is the Hermite form written with the sound speed c_s^2 = 1/3,
the TRT split uses an explicit permutation matrix, and streaming is a pull
through ``np.roll`` on 3-D arrays. Only suitable for tiny lattices.
"""
from __future__ import annotations

import itertools

import numpy as np

CS2 = 1.0 / 3.0


def d3q19():
    """Velocities (all c in {-1,0,1}^3 with |c|^2 <= 2) and weights solved from
    sum w = 1, sum w c_x^2 = c_s^2, sum w c_x^2 c_y^2 = c_s^4 (one weight per shell)."""
    cs = [c for c in itertools.product((-1, 0, 1), repeat=3) if sum(v * v for v in c) <= 2]
    cs = np.array(cs, dtype=np.int64)
    shell = (cs * cs).sum(1)
    A = np.zeros((3, 3))
    b = np.array([1.0, CS2, CS2 * CS2])
    for s in range(3):
        m = shell == s
        A[0, s] = m.sum()
        A[1, s] = (cs[m, 0] ** 2).sum()
        A[2, s] = (cs[m, 0] ** 2 * cs[m, 1] ** 2).sum()
    w_shell = np.linalg.solve(A, b)
    return cs, w_shell[shell]


C, W = d3q19()
NQ = C.shape[0]
OPP = np.array([int(np.nonzero((C == -C[i]).all(1))[0][0]) for i in range(NQ)])
PERM = np.zeros((NQ, NQ))
PERM[np.arange(NQ), OPP] = 1.0


def equilibrium(rho, u):
    """rho [...], u [3, ...] -> [19, ...]."""
    cu = np.einsum("qa,a...->q...", C.astype(float), u)
    uu = (u * u).sum(0)
    return W.reshape((-1,) + (1,) * rho.ndim) * rho * (
        1.0 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu / (2 * CS2))


def collide(f, omega_p, omega_m, F):
    """TRT + simple body-force source w_i (c_i . F) / c_s^2 on f [19, ...]."""
    rho = f.sum(0)
    j = np.einsum("qa,q...->a...", C.astype(float), f)
    with np.errstate(invalid="ignore", divide="ignore"):
        e = equilibrium(rho, j / rho)   # 0/0 only at half-way solid cells, masked by the caller
    fo = np.einsum("pq,q...->p...", PERM, f)
    eo = np.einsum("pq,q...->p...", PERM, e)
    fplus, fminus = (f + fo) / 2, (f - fo) / 2
    eplus, eminus = (e + eo) / 2, (e - eo) / 2
    src = (W * (C.astype(float) @ np.asarray(F, dtype=float)) / CS2).reshape((-1,) + (1,) * rho.ndim)
    return f - omega_p * (fplus - eplus) - omega_m * (fminus - eminus) + src


def step_pull(fq, flags, omega_p, omega_m, F):
    """fq: [19, nz, ny, nx] post-streaming PDFs; flags [nz, ny, nx].

    Post-collision state everywhere (full-way solid: reversal, half-way solid: 0),
    then every direction is pulled from its upstream neighbour; a link whose
    upstream cell is half-way solid takes the local reflected population."""
    fluid = flags == 0
    full = flags == 1
    post = np.zeros_like(fq)
    coll = collide(fq, omega_p, omega_m, F)
    post[:, fluid] = coll[:, fluid]
    post[:, full] = fq[OPP][:, full]
    out = np.zeros_like(fq)
    half = flags == 2
    for i in range(NQ):
        cx, cy, cz = C[i]
        pulled = np.roll(post[i], shift=(cz, cy, cx), axis=(0, 1, 2))
        upstream_half = np.roll(half, shift=(cz, cy, cx), axis=(0, 1, 2))
        val = np.where(upstream_half, post[OPP[i]], pulled)
        out[i] = np.where(half, 0.0, val)
    return out


def to_reference_order(f_oracle, c_oracle):
    """Permute a [19, ...] array from another velocity order into this one."""
    perm = [int(np.nonzero((c_oracle == C[i]).all(1))[0][0]) for i in range(NQ)]
    return f_oracle[perm]
