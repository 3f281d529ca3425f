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


def krylov_kernel(dens, K0, rank, f=None, rel_tol=None, breakdown=1e-12):
    """Low-rank K f for the density `dens` (an electronic.Density).

    rank:     maximum number of directions m.
    rel_tol:  optional adaptive stop: after each direction, stop once
              |F~ c - f~| / |f~| < rel_tol (the SCF's "2-3 ranks adaptively").
    Returns (Kf, info) with info holding V, F~, c and the relative LSQ
    residual."""
    if f is None:
        f = dens.residual()
    ft = K0 @ f
    nft = np.linalg.norm(ft)
    V, FT = [], []
    c = np.zeros(0)
    rel = 1.0
    w = ft.copy()
    for k in range(rank):
        for _ in range(2):
            for v in V:
                w = w - (v @ w) * v
        nw = np.linalg.norm(w)
        if nw <= breakdown * max(nft, 1e-300):
            break
        v = w / nw
        fv = dens.fv(v)
        V.append(v)
        FT.append(K0 @ fv)
        Fm = np.array(FT).T
        c = np.linalg.lstsq(Fm, ft, rcond=None)[0]
        rel = np.linalg.norm(Fm @ c - ft) / max(nft, 1e-300)
        if rel_tol is not None and rel < rel_tol:
            break
        w = FT[-1].copy()
    if not V:
        return np.zeros_like(f), dict(V=np.zeros((f.size, 0)), FT=np.zeros((f.size, 0)),
                                      c=c, rel=rel, rank=0)
    Vm = np.array(V).T
    return Vm @ c, dict(V=Vm, FT=np.array(FT).T, c=c, rel=rel, rank=len(V))


def exact_kernel(dens):
    """K = J^{-1} from the full Jacobian (the exact t0 preconditioner)."""
    return np.linalg.inv(dens.jacobian())
