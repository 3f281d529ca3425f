"""Python binding of libsxl.so (include/sxl.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module only
checks shapes, passes device pointers of torch tensors and the stream, and
turns status codes into exceptions.  Importing it does not need a GPU;
creating a Context does, and fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsxl.so")

FP64, MIXED_FP16, MIXED_BF16 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp16": MIXED_FP16, "bf16": MIXED_BF16}
K0_MINUS_IDENTITY, K0_GIVEN = 0, 1

_d = ctypes.c_double
_i = ctypes.c_int
_p = ctypes.c_void_p


class Params(ctypes.Structure):
    """Mirror of sxl_params (include/sxl.h)."""
    _fields_ = [
        ("n_atoms", _i), ("cell", _d * 3),
        ("eps_s", _d), ("eps_p", _d), ("eps_d", _d),
        ("V0", _d * 10),
        ("q_decay", _d), ("r0", _d), ("r_cut", _d), ("r_on", _d),
        ("U", _d), ("W", _d), ("coulomb_k", _d),
        ("kT", _d), ("n_elec_per_atom", _d),
        ("d0_s", _d), ("d0_p", _d), ("d0_d", _d),
        ("rep_A", _d), ("rep_b", _d),
        ("mass_amu", _d), ("dt_fs", _d),
        ("krylov_rank", _i), ("kmax", _i),
        ("kappa", _d), ("alpha", _d), ("c", _d * 10),
        ("precision", _i), ("foe_steps", _i), ("foe_u_max", _d),
        ("mu_max_iter", _i), ("mu_tol", _d), ("scf_keep_k0", _i),
        ("S0", _d * 10), ("s_decay", _d), ("l_resolved", _i), ("J_l", _d * 3),
        ("krylov_recycle", _i),
    ]


MIXERS = {"kernel": 0, "linear": 1, "diis": 2}


class ScfOpts(ctypes.Structure):
    """Mirror of sxl_scf_opts (include/sxl.h)."""
    _fields_ = [("mixer", _i), ("lin_mix", _d), ("switch_rms", _d), ("diis_hist", _i),
                ("diis_mix", _d), ("krylov_rel_tol", _d)]


EXPORTS = {
    "sxl_create": (_i, [ctypes.POINTER(Params), _p, ctypes.POINTER(_p)]),
    "sxl_destroy": (_i, [_p]),
    "sxl_last_error": (ctypes.c_char_p, [_p]),
    "sxl_hamiltonian": (_i, [_p, _p, _p, _p]),
    "sxl_density": (_i, [_p, _p, _p, _p, ctypes.POINTER(_d)]),
    "sxl_density_matrix": (_i, [_p, _p]),
    "sxl_response": (_i, [_p, _p, _p, ctypes.POINTER(_d)]),
    "sxl_set_k0": (_i, [_p, _i, _p]),
    "sxl_build_exact_k0": (_i, [_p, _p]),
    "krylov_kernel_apply": (_i, [_p, _p, _p, _i, _p, _p, ctypes.POINTER(_d)]),
    "forces": (_i, [_p, _p, _p, _p, _p]),
    "sxl_set_state": (_i, [_p, _p, _p, _p, _d]),
    "sxl_get_state": (_i, [_p, _p, _p, _p, ctypes.POINTER(_d)]),
    "sxl_set_state_host": (_i, [_p, _p, _p, _p, _d]),
    "sxl_get_state_host": (_i, [_p, _p, _p, _p, ctypes.POINTER(_d)]),
    "xlbomd_step": (_i, [_p, _i, _p]),
    "scf_solve": (_i, [_p, _p, _p, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "scf_solve_ex": (_i, [_p, _p, _p, _d, _i, ctypes.POINTER(ScfOpts), _p, ctypes.POINTER(_i),
                          ctypes.POINTER(_d)]),
    "bomd_step": (_i, [_p, _i, ctypes.POINTER(ScfOpts), _d, _i, _p, _p]),
    "sxl_batch_create": (_i, [ctypes.POINTER(Params), _i, ctypes.POINTER(_p)]),
    "sxl_batch_context": (_i, [_p, _i, ctypes.POINTER(_p)]),
    "sxl_batch_step": (_i, [_p, _i, _i, _p]),
    "sxl_batch_destroy": (_i, [_p]),
    "sxl_info": (_i, [_p, _p]),
    "sxl_mixed_gemm": (_i, [_p, _p, _p, _p, _p, _d, _d, _d, _i, _i]),
    "sxl_set_derived_host": (_i, [_p, _p, _p]),
    "sxl_get_derived_host": (_i, [_p, _p, _p]),
    "sxl_get_charges_host": (_i, [_p, _p]),
    "sxl_checkpoint_write": (_i, [_p, ctypes.c_char_p]),
    "sxl_checkpoint_read": (_i, [_p, ctypes.c_char_p]),
    "sxl_md_step": (ctypes.c_longlong, [_p]),
    "sxl_selftest_timeout": (_i, [_p, _d]),
    "krylov_kernel_subspace": (_i, [_p, _p, _p, _p, _i, _i, _i, _p, _p, _p]),
    "sxl_timers": (_i, [_p, _p, _i]),
    "sxl_enable_gemm_timing": (_i, [_p, _i]),
    "sxl_gemm_timers": (_i, [_p, _p, _i]),
    "sxl_gemm_f64": (_i, [_p, _p, _p, _p, _p, _d, _d, _d, _i]),
    "sxl_autotune": (_i, [_p, _p]),
    "sxl_set_tiles": (_i, [_p, _i, _i, _i, _i]),
    "sxl_set_product_kernel": (_i, [_p, _i]),
    "sxl_mixed_gemm_fused": (_i, [_p, _i, _p, _i, _p, _i, _p, _p, _d, _d, _d, _i, _i]),
    "sxl_batch_autotune": (_i, [_p, _p]),
    "sxl_mixed_gemm_noalloc": (_i, [_i, _i, _p, _p, _p, _p, _d, _d, _d, _i, _i, _p]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libsxl.so and declares the C signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsxl.so not found at {path}: run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class SxlError(RuntimeError):
    """A library call returned a negative status; .code holds it (SXL_E_*)."""

    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


# status codes of include/sxl.h
E_ARG, E_CUDA, E_NOMEM, E_NO_CONVERGENCE, E_NAN, E_STATE, E_UNSUPPORTED, E_TIMEOUT, E_IO = \
    -1, -2, -3, -4, -5, -6, -7, -8, -9


def make_params(mp, n_atoms: int, cell, precision="fp64", foe_steps=0, foe_u_max=0.0,
                mu_tol=0.0, mu_max_iter=0, scf_keep_k0=0, krylov_recycle=0) -> Params:
    """Params from a workload.ModelParams-like object."""
    p = Params()
    p.n_atoms = int(n_atoms)
    p.cell[:] = [float(x) for x in cell]
    p.eps_s, p.eps_p, p.eps_d = mp.eps_s, mp.eps_p, mp.eps_d
    p.V0[:] = [float(x) for x in mp.V0]
    p.q_decay, p.r0, p.r_cut, p.r_on = mp.q_decay, mp.r0, mp.r_cut, mp.r_on
    p.U, p.W, p.coulomb_k = mp.U, mp.W, mp.coulomb_k
    p.kT, p.n_elec_per_atom = mp.kT, mp.n_elec_per_atom
    p.d0_s, p.d0_p, p.d0_d = mp.d0_s, mp.d0_p, mp.d0_d
    p.rep_A, p.rep_b = mp.rep_A, mp.rep_b
    p.mass_amu, p.dt_fs = mp.mass_amu, mp.dt_fs
    p.krylov_rank, p.kmax = int(mp.krylov_rank), int(mp.kmax)
    p.kappa, p.alpha = mp.kappa, mp.alpha
    cc = list(mp.c) + [0.0] * (10 - len(mp.c))
    p.c[:] = [float(x) for x in cc]
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.foe_steps = int(foe_steps)
    p.foe_u_max = float(foe_u_max)
    p.mu_max_iter = int(mu_max_iter)
    p.mu_tol = float(mu_tol)
    p.scf_keep_k0 = int(scf_keep_k0)
    p.S0[:] = [float(x) for x in getattr(mp, "S0", (0.0,) * 10)]
    p.s_decay = float(getattr(mp, "s_decay", mp.q_decay))
    p.l_resolved = int(bool(getattr(mp, "l_resolved", False)))
    p.J_l[:] = [float(x) for x in getattr(mp, "J_l", (0.5 * mp.W,) * 3)]
    p.krylov_recycle = int(krylov_recycle)
    return p


def _ptr(t, n=None, name="array"):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
        raise TypeError(f"{name} must be a float64 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One library context (device buffers, stream, MD state)."""

    def __init__(self, mp, n_atoms: int, cell, precision="fp64", stream=None, **kw):
        import torch
        self.lib = load_library()
        self.nat = int(n_atoms)
        self.N = 9 * self.nat
        # extended-vector length: per atom, or per (atom, shell) when l-resolved
        self.n2 = 2 * self.nat * (3 if getattr(mp, "l_resolved", False) else 1)
        self.kmax = int(mp.kmax)
        self.params = make_params(mp, n_atoms, cell, precision, **kw)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _p()
        rc = self.lib.sxl_create(ctypes.byref(self.params), _p(self.stream.cuda_stream),
                                 ctypes.byref(h))
        if rc != 0:
            raise SxlError(f"sxl_create failed with code {rc}")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.sxl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != 0:
            msg = self.lib.sxl_last_error(self.h).decode()
            raise SxlError(f"{what} failed ({rc}): {msg}", rc)

    def _dev(self, x):
        import torch
        if isinstance(x, torch.Tensor):
            return x.to(device="cuda", dtype=torch.float64).contiguous()
        return torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda").contiguous()

    def _new(self, *shape):
        import torch
        return torch.empty(*shape, dtype=torch.float64, device="cuda")

    # -- stages -------------------------------------------------------------
    def hamiltonian(self, R, n, want_H=True):
        R, n = self._dev(R), self._dev(n)
        H = self._new(2, self.N, self.N) if want_H else None
        self._check(self.lib.sxl_hamiltonian(self.h, _ptr(R, 3 * self.nat), _ptr(n, self.n2),
                                             _ptr(H)), "sxl_hamiltonian")
        return H

    def density(self, R, n, mu: Optional[float] = None):
        R, n = self._dev(R), self._dev(n)
        q = self._new(self.n2)
        m = _d(float("nan") if mu is None else float(mu))
        self._check(self.lib.sxl_density(self.h, _ptr(R, 3 * self.nat), _ptr(n, self.n2),
                                         _ptr(q), ctypes.byref(m)), "sxl_density")
        return q, m.value

    def density_matrix(self):
        D = self._new(2, self.N, self.N)
        self._check(self.lib.sxl_density_matrix(self.h, _ptr(D)), "sxl_density_matrix")
        return D

    def response(self, v):
        v = self._dev(v)
        qv = self._new(self.n2)
        dmu = _d(0.0)
        self._check(self.lib.sxl_response(self.h, _ptr(v, self.n2), _ptr(qv), ctypes.byref(dmu)),
                    "sxl_response")
        return qv, dmu.value

    def set_k0(self, K0=None):
        if K0 is None:
            self._check(self.lib.sxl_set_k0(self.h, K0_MINUS_IDENTITY, None), "sxl_set_k0")
        else:
            K0 = self._dev(K0)
            self._check(self.lib.sxl_set_k0(self.h, K0_GIVEN, _ptr(K0, self.n2 * self.n2)),
                        "sxl_set_k0")

    def build_exact_k0(self, want_J=False):
        J = self._new(self.n2, self.n2) if want_J else None
        self._check(self.lib.sxl_build_exact_k0(self.h, _ptr(J)), "sxl_build_exact_k0")
        return J

    def krylov(self, R, n, rank):
        R, n = self._dev(R), self._dev(n)
        Kf, q = self._new(self.n2), self._new(self.n2)
        rel = _d(0.0)
        self._check(self.lib.krylov_kernel_apply(self.h, _ptr(R, 3 * self.nat), _ptr(n, self.n2),
                                                 int(rank), _ptr(Kf), _ptr(q), ctypes.byref(rel)),
                    "krylov_kernel_apply")
        return Kf, q, rel.value

    def forces(self, R, n, energies=True):
        R, n = self._dev(R), self._dev(n)
        F = self._new(self.nat, 3)
        en = (ctypes.c_double * 6)() if energies else None
        self._check(self.lib.forces(self.h, _ptr(R, 3 * self.nat), _ptr(n, self.n2), _ptr(F),
                                    en), "forces")
        if not energies:
            return F, None
        keys = ("U", "band", "coul", "spin", "entropy", "rep")
        return F, dict(zip(keys, list(en)))

    # -- MD -----------------------------------------------------------------
    def set_state(self, R, V, nhist, mu):
        R, V, nh = self._dev(R), self._dev(V), self._dev(nhist)
        self._check(self.lib.sxl_set_state(self.h, _ptr(R, 3 * self.nat), _ptr(V, 3 * self.nat),
                                           _ptr(nh, (self.kmax + 1) * self.n2), float(mu)),
                    "sxl_set_state")

    def get_state(self):
        R, V = self._new(self.nat, 3), self._new(self.nat, 3)
        nh = self._new(self.kmax + 1, self.n2)
        mu = _d(0.0)
        self._check(self.lib.sxl_get_state(self.h, _ptr(R), _ptr(V), _ptr(nh), ctypes.byref(mu)),
                    "sxl_get_state")
        return R, V, nh, mu.value

    def set_state_host(self, R, V, nhist, mu):
        """Host-pointer variant: R, V, nhist are C-contiguous float64 numpy arrays
        (pinned torch CPU tensors also work)."""
        ptrs = [_host_ptr(a) for a in (R, V, nhist)]
        self._check(self.lib.sxl_set_state_host(self.h, *ptrs, float(mu)), "sxl_set_state_host")

    def get_state_host(self, R, V, nhist):
        mu = _d(0.0)
        ptrs = [_host_ptr(a) for a in (R, V, nhist)]
        self._check(self.lib.sxl_get_state_host(self.h, *ptrs, ctypes.byref(mu)),
                    "sxl_get_state_host")
        return mu.value

    def step(self, nsteps=1, stats=True):
        out = np.zeros((max(nsteps, 1), 4)) if stats else None
        ptr = out.ctypes.data_as(_p) if stats else None
        self._check(self.lib.xlbomd_step(self.h, int(nsteps), ptr), "xlbomd_step")
        return out

    def scf(self, R, n, tol=1e-8, max_iter=300):
        R = self._dev(R)
        n = self._dev(n).clone()
        it, rms = _i(0), _d(0.0)
        self._check(self.lib.scf_solve(self.h, _ptr(R, 3 * self.nat), _ptr(n, self.n2),
                                       float(tol), int(max_iter), ctypes.byref(it),
                                       ctypes.byref(rms)), "scf_solve")
        return n, it.value, rms.value

    @staticmethod
    def _scf_opts(mixer="kernel", lin_mix=0.0, switch_rms=0.0, diis_hist=0, diis_mix=0.0,
                  krylov_rel_tol=0.0):
        return ScfOpts(MIXERS[mixer], float(lin_mix), float(switch_rms), int(diis_hist),
                       float(diis_mix), float(krylov_rel_tol))

    def scf_ex(self, R, n, tol=1e-8, max_iter=300, mixer="kernel", **opts):
        """SCF with a choice of mixer ("kernel", "linear", "diis"); returns
        (n, iterations, final RMS, RMS history as a numpy array)."""
        R = self._dev(R)
        n = self._dev(n).clone()
        it, rms = _i(0), _d(0.0)
        hist = np.zeros(int(max_iter))
        o = self._scf_opts(mixer, **opts)
        self._check(self.lib.scf_solve_ex(self.h, _ptr(R, 3 * self.nat), _ptr(n, self.n2),
                                          float(tol), int(max_iter), ctypes.byref(o),
                                          hist.ctypes.data_as(_p), ctypes.byref(it),
                                          ctypes.byref(rms)), "scf_solve_ex")
        return n, it.value, rms.value, hist[:it.value + 1].copy()

    def bomd(self, nsteps=1, tol=1e-6, max_iter=200, mixer="diis", stats=True, **opts):
        """Regular BOMD steps (SCF-converged forces); returns (stats, SCF
        iterations per step)."""
        out = np.zeros((max(nsteps, 1), 4)) if stats else None
        its = np.zeros(max(nsteps, 1), dtype=np.int32)
        o = self._scf_opts(mixer, **opts)
        self._check(self.lib.bomd_step(self.h, int(nsteps), ctypes.byref(o), float(tol),
                                       int(max_iter), out.ctypes.data_as(_p) if stats else None,
                                       its.ctypes.data_as(_p)), "bomd_step")
        return out, its[:nsteps].copy()

    def mixed_gemm(self, A, B, E=None, alpha=1.0, beta=0.0, gamma=0.0, sym=False, split=True):
        """C = alpha A B^T + beta E + gamma I on the tensor-core path (2 x N x N);
        split=True/1 three-product form, False/0 hi parts only, 2 the dual form
        C = alpha (A B^T + B A^T) + beta E + gamma I."""
        A, B = self._dev(A), self._dev(B)
        E = self._dev(E) if E is not None else None
        C = self._new(2, self.N, self.N)
        nn = 2 * self.N * self.N
        self._check(self.lib.sxl_mixed_gemm(self.h, _ptr(A, nn), _ptr(B, nn),
                                            _ptr(E, nn) if E is not None else None, _ptr(C),
                                            float(alpha), float(beta), float(gamma), int(sym),
                                            int(split)), "sxl_mixed_gemm")
        return C

    def mixed_gemm_fused(self, X, Y, m, x_per=True, y_per=True, E=None, alpha=1.0, beta=0.0,
                         gamma=0.0, sym=False, dual=False):
        """Fused products of m right-hand sides (2 m x N x N result); X and Y
        hold 2 m blocks when x_per / y_per, else 2 (one per spin)."""
        X, Y = self._dev(X), self._dev(Y)
        E = self._dev(E) if E is not None else None
        C = self._new(2 * m, self.N, self.N)
        nb = self.N * self.N
        self._check(self.lib.sxl_mixed_gemm_fused(
            self.h, int(m), _ptr(X, (2 * m if x_per else 2) * nb), int(x_per),
            _ptr(Y, (2 * m if y_per else 2) * nb), int(y_per),
            _ptr(E, 2 * m * nb) if E is not None else None, _ptr(C), float(alpha), float(beta),
            float(gamma), int(sym), int(dual)), "sxl_mixed_gemm_fused")
        return C

    def autotune(self):
        """Times the candidate tensor-core tiles on this context and keeps the
        fastest; returns the choice and the times (ms)."""
        out = np.zeros(9)
        self._check(self.lib.sxl_autotune(self.h, out.ctypes.data_as(_p)), "sxl_autotune")
        return {"plain_bk": int(out[0]), "plain_rows": 128 * int(out[1]), "plain_ms": out[2],
                "split_bk": int(out[3]), "split_ms": out[4], "dual_rows": 128 * int(out[5]),
                "dual_ms": out[6], "plain_persistent": bool(out[7]),
                "dual_persistent": bool(out[8])}

    def set_tiles(self, bk_plain=0, mt_plain=0, bk_split=0, mt_dual=0):
        self._check(self.lib.sxl_set_tiles(self.h, int(bk_plain), int(mt_plain), int(bk_split),
                                           int(mt_dual)), "sxl_set_tiles")

    def set_product_kernel(self, kernel="default"):
        """Kernel of the plain and dual products: "persistent", "single" or
        "default"."""
        code = {"default": 0, "persistent": 1, "single": 2}[kernel]
        self._check(self.lib.sxl_set_product_kernel(self.h, code), "sxl_set_product_kernel")

    def gemm_f64(self, A, B, E=None, alpha=1.0, beta=0.0, gamma=0.0, sym=False):
        """C = alpha A B^T + beta E + gamma I in fp64 (2 x N x N), the fp64
        form's product."""
        A, B = self._dev(A), self._dev(B)
        E = self._dev(E) if E is not None else None
        C = self._new(2, self.N, self.N)
        nn = 2 * self.N * self.N
        self._check(self.lib.sxl_gemm_f64(self.h, _ptr(A, nn), _ptr(B, nn),
                                          _ptr(E, nn) if E is not None else None, _ptr(C),
                                          float(alpha), float(beta), float(gamma), int(sym)),
                    "sxl_gemm_f64")
        return C

    def set_derived_host(self, F, Kf):
        self._check(self.lib.sxl_set_derived_host(self.h, _host_ptr(F), _host_ptr(Kf)),
                    "sxl_set_derived_host")

    def get_derived_host(self, F, Kf):
        self._check(self.lib.sxl_get_derived_host(self.h, _host_ptr(F), _host_ptr(Kf)),
                    "sxl_get_derived_host")

    def enable_gemm_timing(self, on=True):
        self._check(self.lib.sxl_enable_gemm_timing(self.h, int(on)), "sxl_enable_gemm_timing")

    def timers(self, reset=False):
        out = np.zeros(10)
        self._check(self.lib.sxl_timers(self.h, out.ctypes.data_as(_p), int(reset)), "sxl_timers")
        keys = ("steps", "density_ms", "forces_ms", "krylov_ms", "ranks", "tc_launches",
                "tc_ms", "tc_mma_flops", "tc_alg_flops", "tc_fp32_flops")
        return dict(zip(keys, out.tolist()))

    def gemm_timers(self, reset=False):
        """Per product form ("plain", "dual", "split", "fp64"): launches, ms,
        issued_flops, product_flops (each product counted once)."""
        out = np.zeros(16)
        self._check(self.lib.sxl_gemm_timers(self.h, out.ctypes.data_as(_p), int(reset)),
                    "sxl_gemm_timers")
        keys = ("launches", "ms", "issued_flops", "product_flops")
        return {name: dict(zip(keys, out[4 * v:4 * v + 4].tolist()))
                for v, name in enumerate(("plain", "dual", "split", "fp64"))}

    def krylov_subspace(self, R, n, cand, rank, fused=True):
        """The recycled-subspace kernel at (R, n) with explicit candidate
        directions (k x n2, or None); returns (Kf, rel, directions kept)."""
        R, n = self._dev(R), self._dev(n)
        cand = self._dev(cand) if cand is not None and len(cand) else None
        k = 0 if cand is None else int(cand.shape[0])
        Kf = self._new(self.n2)
        rel, rk = _d(0.0), _i(0)
        self._check(self.lib.krylov_kernel_subspace(
            self.h, _ptr(R, 3 * self.nat), _ptr(n, self.n2),
            _ptr(cand, k * self.n2) if cand is not None else None, k, int(rank), int(fused),
            _ptr(Kf), ctypes.byref(rel), ctypes.byref(rk)), "krylov_kernel_subspace")
        return Kf, rel.value, rk.value

    def charges(self):
        """q of the last evaluation at the context state (numpy, n2)."""
        out = np.zeros(self.n2)
        self._check(self.lib.sxl_get_charges_host(self.h, out.ctypes.data_as(_p)),
                    "sxl_get_charges_host")
        return out

    def checkpoint_write(self, path):
        self._check(self.lib.sxl_checkpoint_write(self.h, os.fsencode(path)),
                    "sxl_checkpoint_write")

    def checkpoint_read(self, path):
        self._check(self.lib.sxl_checkpoint_read(self.h, os.fsencode(path)),
                    "sxl_checkpoint_read")

    def md_step(self):
        return int(self.lib.sxl_md_step(self.h))

    def selftest_timeout(self, seconds=0.25):
        """Runs the bounded-wait self-test; raises SxlError with code
        E_TIMEOUT, as a tensor-core GEMM barrier timeout would."""
        self._check(self.lib.sxl_selftest_timeout(self.h, float(seconds)),
                    "sxl_selftest_timeout")

    def info(self):
        out = np.zeros(7)
        self._check(self.lib.sxl_info(self.h, out.ctypes.data_as(_p)), "sxl_info")
        keys = ("mu", "N", "foe_steps", "lam_min", "lam_max", "gemms", "launches")
        return dict(zip(keys, out.tolist()))


def _make_autograd():
    import torch

    class ShadowEnergy(torch.autograd.Function):
        """U(R) at constant n (Eq. ShadowULatte) with dU/dR from the library.

        forward(R, n, ctx) runs the density and the force kernel of
        sxl_forces: the force kernel is the adjoint of the energy with
        respect to the positions (Tr[D dH0/dR] with the Slater-Koster
        derivative blocks formed on the fly from the density matrix of the
        expansion chain, plus the Coulomb and repulsion terms; the spin and
        entropy terms have no explicit R dependence at constant n and the
        density is stationary).  backward returns -F times the incoming
        gradient; no per-orbital derivative tensor is ever stored.
        """

        @staticmethod
        def forward(fctx, R, n, ctx):
            F, en = ctx.forces(R.detach(), n.detach(), energies=True)
            fctx.save_for_backward(F)
            return torch.tensor(en["U"], dtype=torch.float64, device=R.device)

        @staticmethod
        def backward(fctx, gU):
            (F,) = fctx.saved_tensors
            return (-F * gU).reshape(F.shape), None, None

    return ShadowEnergy


_SHADOW = None


def shadow_energy(R, n, ctx):
    """Differentiable shadow energy: U = shadow_energy(R, n, ctx);
    U.backward() fills R.grad with dU/dR = -F (eV/Angstrom)."""
    global _SHADOW
    if _SHADOW is None:
        _SHADOW = _make_autograd()
    return _SHADOW.apply(R, n, ctx)


def mixed_gemm_noalloc(n, precision, A, B, E=None, alpha=1.0, beta=0.0, gamma=0.0,
                       sym=False, split=True, stream=None):
    """Allocation-free tensor-core product (sxl_mixed_gemm_noalloc): the caller
    passes A, B, E and receives C (2 x n x n fp64 CUDA tensors)."""
    import torch
    lib = load_library()
    nn = 2 * n * n
    dev = A.device
    for name, t in (("B", B), ("E", E)):
        if t is not None and t.device != dev:
            raise ValueError(f"{name} is on {t.device}, A on {dev}: all operands must share a device")
    # the library works on the current device (its scratch and the stream's)
    with torch.cuda.device(dev):
        C = torch.empty(2, n, n, dtype=torch.float64, device=dev)
        st = stream if stream is not None else torch.cuda.current_stream(dev)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        rc = lib.sxl_mixed_gemm_noalloc(int(n), prec, _ptr(A, nn), _ptr(B, nn),
                                        _ptr(E, nn) if E is not None else None, _ptr(C),
                                        float(alpha), float(beta), float(gamma), int(sym),
                                        int(split), _p(st.cuda_stream))
    if rc != 0:
        raise SxlError(f"sxl_mixed_gemm_noalloc failed ({rc})")
    return C


def _host_ptr(a):
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("host arrays must be contiguous float64 CPU tensors")
        return _p(a.data_ptr())
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data_as(_p)


class _BatchContext(Context):
    """A replica of a Batch: the context lives on a stream the batch owns, so
    every call is bracketed by device synchronization (setup and inspection,
    not the batched step)."""

    def __init__(self, batch, handle, mp, n_atoms, cell, precision):
        import torch
        self.lib = batch.lib
        self.nat = int(n_atoms)
        self.N = 9 * self.nat
        # extended-vector length: per atom, or per (atom, shell) when l-resolved
        self.n2 = 2 * self.nat * (3 if getattr(mp, "l_resolved", False) else 1)
        self.kmax = int(mp.kmax)
        self.params = make_params(mp, n_atoms, cell, precision)
        self.stream = torch.cuda.current_stream()
        self.h = handle
        self._owned = False

    def _dev(self, x):
        import torch
        t = super()._dev(x)
        torch.cuda.synchronize()
        return t

    def _check(self, rc, what):
        import torch
        torch.cuda.synchronize()
        super()._check(rc, what)

    def close(self):
        self.h = None   # owned by the batch


class Batch:
    """Independent replicas (any sizes) stepped together: one context per
    replica on its own stream, driven by a pool of host threads."""

    def __init__(self, workloads, precision="fp16", **kw):
        self.lib = load_library()
        self.workloads = list(workloads)
        arr = (Params * len(self.workloads))()
        for i, w in enumerate(self.workloads):
            arr[i] = make_params(w.params, w.R.shape[0], w.cell, precision, **kw)
        h = _p()
        rc = self.lib.sxl_batch_create(arr, len(self.workloads), ctypes.byref(h))
        if rc != 0:
            raise SxlError(f"sxl_batch_create failed with code {rc}")
        self.h = h
        self.contexts = []
        for i, w in enumerate(self.workloads):
            c = _p()
            if self.lib.sxl_batch_context(self.h, i, ctypes.byref(c)) != 0:
                raise SxlError("sxl_batch_context failed")
            self.contexts.append(_BatchContext(self, c, w.params, w.R.shape[0], w.cell, precision))

    def autotune(self):
        """Tile autotuning of every replica (one run per distinct chain
        dimension); returns one dict per tuned dimension."""
        rep = np.zeros((len(self.contexts), 10))
        k = self.lib.sxl_batch_autotune(self.h, rep.ctypes.data_as(_p))
        if k < 0:
            raise SxlError(f"sxl_batch_autotune failed ({k})")
        keys = ("n", "plain_bk", "plain_mt", "plain_ms", "split_bk", "split_ms", "dual_mt",
                "dual_ms", "plain_persistent", "dual_persistent")
        return [dict(zip(keys, r.tolist())) for r in rep[:k]]

    def step(self, nsteps=1, nthreads=0):
        """nsteps sXL-BOMD steps of every replica; returns the per-replica
        status codes (raises if any is not 0)."""
        status = np.zeros(len(self.contexts), dtype=np.int32)
        rc = self.lib.sxl_batch_step(self.h, int(nsteps), int(nthreads), status.ctypes.data_as(_p))
        if rc != 0:
            bad = [i for i, s in enumerate(status) if s != 0]
            msgs = [self.lib.sxl_last_error(self.contexts[i].h).decode() for i in bad[:3]]
            raise SxlError(f"sxl_batch_step failed ({rc}) for replicas {bad}: {msgs}")
        return status

    def close(self):
        if getattr(self, "h", None):
            self.lib.sxl_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
