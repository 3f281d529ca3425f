"""Oracle: the preconditioned low-rank Krylov approximation of the kernel
(Sec. II.G, Eqs. fv, mIJacobian).

Test infrastructure only (see oracle/__init__.py).

With f = q[n] - n and a preconditioner K0 ~ J^{-1}:
  f~ = K0 f;  directions v_k are an orthonormal basis of the Krylov space
  span{f~, (K0 J) f~, (K0 J)^2 f~, ...}, built one vector at a time: the next
  candidate is f~_{v_k} = K0 f_{v_k} = K0 J v_k, orthogonalized against the
  previous v's (two passes of modified Gram-Schmidt) and normalized.
  With orthonormal v, O = I and L = I, and Eq. mIJacobian gives
  (K0 J)^{-1} f~ ~ sum_{k,l} v_k M_kl f~_{v_l}^T f~ with M = (F~^T F~)^{-1},
  i.e. K f ~ V c where c solves the least-squares problem min |F~ c - f~|.
Newton's step for f(n) = 0 is -J^{-1} f, so K f ~ J^{-1} f and
n'' = -w^2 K f (Eq. Eq_Mot2); the SCF update of Eq. QN is n - K f.
"""
from __future__ import annotations

import numpy as np


class KrylovBuilder:
    """The Krylov loop of Eq. mIJacobian one direction at a time, so that a
    caller can time or inspect every direction (each needs one response).

    add_direction() orthogonalizes the current candidate against the previous
    v's (two passes of modified Gram-Schmidt), normalizes it, takes its
    response f~_v = K0 (q_v - v) and solves min |F~ c - f~|; it returns False
    at breakdown (the candidate is numerically inside the span)."""

    def __init__(self, dens, K0, f=None, breakdown=1e-12):
        self.dens, self.K0, self.breakdown = dens, K0, breakdown
        self.f = dens.residual() if f is None else f
        self.ft = K0 @ self.f
        self.nft = np.linalg.norm(self.ft)
        self.V, self.FT = [], []
        self.c = np.zeros(0)
        self.rel = 1.0
        self.w = self.ft.copy()

    def add_direction(self):
        w = self.w
        for _ in range(2):
            for v in self.V:
                w = w - (v @ w) * v
        nw = np.linalg.norm(w)
        if nw <= self.breakdown * max(self.nft, 1e-300):
            return False
        v = w / nw
        fv = self.dens.fv(v)
        self.V.append(v)
        self.FT.append(self.K0 @ fv)
        Fm = np.array(self.FT).T
        self.c = np.linalg.lstsq(Fm, self.ft, rcond=None)[0]
        self.rel = np.linalg.norm(Fm @ self.c - self.ft) / max(self.nft, 1e-300)
        self.w = self.FT[-1].copy()
        return True

    def result(self):
        """(K f ~ V c, info) for the directions added so far."""
        f = self.f
        if not self.V:
            return np.zeros_like(f), dict(V=np.zeros((f.size, 0)), FT=np.zeros((f.size, 0)),
                                          c=self.c, rel=self.rel, rank=0)
        Vm = np.array(self.V).T
        return Vm @ self.c, dict(V=Vm, FT=np.array(self.FT).T, c=self.c, rel=self.rel,
                                 rank=len(self.V))


def krylov_kernel(dens, K0, rank, f=None, rel_tol=None, breakdown=1e-12):
    """Low-rank K f for the density `dens` (an electronic.Density).

    rank:     maximum number of directions m.
    rel_tol:  optional adaptive stop: after each direction, stop once
              |F~ c - f~| / |f~| < rel_tol (the SCF's "2-3 ranks adaptively").
    Returns (Kf, info) with info holding V, F~, c and the relative LSQ
    residual."""
    kb = KrylovBuilder(dens, K0, f=f, breakdown=breakdown)
    for _ in range(rank):
        if not kb.add_direction():
            break
        if rel_tol is not None and kb.rel < rel_tol:
            break
    return kb.result()


def exact_kernel(dens):
    """K = J^{-1} from the full Jacobian (the exact t0 preconditioner)."""
    return np.linalg.inv(dens.jacobian())


def krylov_kernel_subspace(dens, K0, candidates, rank, f=None, drop=1e-6):
    """Recycled-subspace variant of the low-rank kernel (a build choice, not
    the paper's construction): the directions are not generated one
    response at a time but taken from a given list.

    directions: f~ = K0 f first, then the candidates in order, each
                orthogonalized against the directions kept so far (two
                passes of modified Gram-Schmidt) and kept when its norm
                after that is above `drop` times its norm before; at most
                `rank` directions;
    responses:  f~_v = K0 (q_v - v) for every kept v (independent of one
                another, so they can be computed together);
    kernel:     c solves min |F~ c - f~|, K f ~ V c (Eq. mIJacobian with
                orthonormal V, as in krylov_kernel).
    With the previous steps' directions as candidates the subspace follows
    the trajectory and every response of a step is known up front.
    Returns (Kf, info) like krylov_kernel."""
    f = dens.residual() if f is None else f
    ft = K0 @ f
    nft = np.linalg.norm(ft)
    V = []
    for w0 in [ft] + [np.asarray(c, dtype=np.float64) for c in candidates]:
        if len(V) == rank:
            break
        w = np.array(w0, dtype=np.float64)
        n0 = np.linalg.norm(w)
        for _ in range(2):
            for v in V:
                w = w - (v @ w) * v
        nw = np.linalg.norm(w)
        if not nw > drop * n0:
            continue
        V.append(w / nw)
    if not V:
        return np.zeros_like(f), dict(V=np.zeros((f.size, 0)), FT=np.zeros((f.size, 0)),
                                      c=np.zeros(0), rel=1.0, rank=0)
    Vm = np.array(V).T
    FT = np.array([K0 @ dens.fv(v) for v in V]).T
    c = np.linalg.lstsq(FT, ft, rcond=None)[0]
    rel = np.linalg.norm(FT @ c - ft) / max(nft, 1e-300)
    return Vm @ c, dict(V=Vm, FT=FT, c=c, rel=rel, rank=len(V))
