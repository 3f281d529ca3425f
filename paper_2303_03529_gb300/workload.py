"""Seeded synthetic inputs for the spin-polarized XL-BOMD hot path.

This module is shared by the CUDA path, the tests and the FP64 oracle. It only
produces inputs: model parameter sets, bcc iron-like cells with Gaussian
displacements, Maxwell velocities and the initial extended charge/spin vector
n. It holds none of the method's arithmetic (no Hamiltonian, no density matrix,
no response, no integrator).

The paper demonstrates the method on a 16-atom bcc Fe supercell (Sec. III.B,
Fig. energy); its real Fe parameters (PLATO integrals, fitted repulsion,
Sec. III.D) are not available, so the workloads here use a synthetic
orthogonal s/p/d Slater-Koster "iron-like" model with the sizes of the
paper's Fe cells scaled up to 128 and 1024 atoms.

Layout conventions used everywhere:
  * positions R: (N_at, 3) float64, Angstrom, atoms ordered lexicographically
    over cells (i, j, k) with the two bcc basis atoms innermost;
  * extended vector n: (2 N_at,) float64, spin-up block first then spin-down
    (Sec. II.G, the 2N-dimensional matrix notation), in electrons relative to
    the neutral atom (4 electrons per spin per atom);
  * velocities: (N_at, 3) float64, Angstrom/fs.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

# Bond-integral order used in every parameter vector V0.
BOND_NAMES = ("sss", "sps", "sds", "pps", "ppp", "pds", "pdp", "dds", "ddp", "ddd")

# Physical constants used only to draw the initial velocities.
KB_EV_PER_K = 8.617333262e-5          # Boltzmann constant, eV/K
AMU_A2_PER_FS2_IN_EV = 103.642696562  # 1 amu * A^2 / fs^2 expressed in eV

SEED_BASE = 2303035290


@dataclasses.dataclass
class ModelParams:
    """Parameters of the synthetic iron-like SCC tight-binding model.

    Units: eV, Angstrom, fs, amu.  Field names follow the C struct
    ``sxl_params`` in include/sxl.h one to one.
    """

    eps_s: float = -3.0
    eps_p: float = 3.0
    eps_d: float = -6.0
    V0: tuple = (-1.5, 1.8, -1.0, 2.5, -0.6, -1.2, 0.5, -0.9, 0.5, -0.08)
    q_decay: float = 1.5      # 1/Angstrom, radial decay of every bond integral
    r0: float = 2.48          # Angstrom, reference bond length
    r_cut: float = 5.0        # Angstrom, hopping cutoff
    r_on: float = 4.5         # Angstrom, start of the smooth switch
    U: float = 4.0            # eV, on-site Hubbard term gamma_II
    W: float = -0.6           # eV, spin coupling (shift +-W s_I / 2)
    coulomb_k: float = 1.0    # eV*Angstrom, prefactor of the screened Coulomb tail
    kT: float = 0.1           # eV, electronic temperature
    n_elec_per_atom: float = 8.0
    # neutral-atom occupations per spin and orbital (s, each p, each d)
    d0_s: float = 1.0
    d0_p: float = 0.0
    d0_d: float = 0.6
    # pair repulsion Phi(r) = rep_A exp(-rep_b (r - r0)) s(r); rep_A makes
    # the ideal 4x4x4 bcc cell at a = 2.87 A pressure-free (oracle/fit_repulsion.py)
    rep_A: float = 2.849592917636214
    rep_b: float = 3.0
    mass_amu: float = 55.845
    dt_fs: float = 0.5
    krylov_rank: int = 4
    # dissipative integrator: kappa, alpha, c_0..c_kmax
    kmax: int = 5
    kappa: float = 1.82
    alpha: float = 0.018
    c: tuple = (-6.0, 14.0, -8.0, -3.0, 4.0, -1.0)
    # paper-general model (Sec. III.A): overlap integrals S0 (same order as
    # V0; all zero = orthogonal basis, S = I) with radial decay s_decay, and
    # l-resolved charges and spins with l-dependent Stoner parameters J_l
    # (s, p, d) in place of the per-atom W / 2
    S0: tuple = (0.0,) * 10
    s_decay: float = 1.5
    l_resolved: bool = False
    J_l: tuple = (-0.3, -0.3, -0.3)

    def replace(self, **kw) -> "ModelParams":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class Workload:
    """One seeded synthetic cell: geometry, velocities, initial n, parameters."""

    name: str
    ncell: int
    a: float
    R: np.ndarray          # (N_at, 3)
    V: np.ndarray          # (N_at, 3)
    n0: np.ndarray         # (2 N_at,)
    cell: np.ndarray       # (3,)
    params: ModelParams
    steps: int
    # the make_cell arguments that regenerate R, V and n0 (see config())
    recipe: Optional[dict] = None
    shell_resolved_n0: bool = False

    @property
    def n_atoms(self) -> int:
        return self.R.shape[0]

    @property
    def n_orb(self) -> int:
        return 9 * self.R.shape[0]


def bcc_positions(ncell: int, a: float) -> np.ndarray:
    """Ideal bcc positions of an ncell^3 cubic supercell, basis atom innermost."""
    out = np.empty((2 * ncell ** 3, 3))
    p = 0
    for i in range(ncell):
        for j in range(ncell):
            for k in range(ncell):
                base = np.array([i, j, k], dtype=np.float64) * a
                out[p] = base
                out[p + 1] = base + 0.5 * a
                p += 2
    return out


def maxwell_velocities(rng: np.random.Generator, n_atoms: int, mass_amu: float,
                       T_K: float) -> np.ndarray:
    """Maxwell-Boltzmann velocities (Angstrom/fs), centre-of-mass momentum
    removed and rescaled to exactly T_K with 3N-3 degrees of freedom."""
    if n_atoms < 2:
        return np.zeros((n_atoms, 3))
    sigma = np.sqrt(KB_EV_PER_K * T_K / (mass_amu * AMU_A2_PER_FS2_IN_EV))
    v = rng.normal(0.0, sigma, size=(n_atoms, 3))
    v -= v.mean(axis=0, keepdims=True)
    ke = 0.5 * mass_amu * AMU_A2_PER_FS2_IN_EV * np.sum(v * v)
    t_now = 2.0 * ke / ((3 * n_atoms - 3) * KB_EV_PER_K)
    v *= np.sqrt(T_K / t_now)
    return v


def initial_n(rng: np.random.Generator, n_atoms: int, m0: float = 2.0,
              noise: float = 0.1) -> np.ndarray:
    """Ferromagnetic start: per-atom spin m_I = m0 + U(-noise, noise), charge 0.

    Returns n = [n_up; n_dn] with n_up = m/2, n_dn = -m/2 (net charge zero)."""
    m = m0 + rng.uniform(-noise, noise, size=n_atoms)
    return np.concatenate([0.5 * m, -0.5 * m])


def make_cell(ncell: int, *, seed: int, sigma: float = 0.05, a: float = 2.87,
              T_K: float = 300.0, params: Optional[ModelParams] = None,
              name: str = "custom", steps: int = 0, m0: float = 2.0,
              noise: float = 0.1, vacancy_frac: float = 0.0) -> Workload:
    """Seeded bcc cell with Gaussian displacements (per component, sigma in A);
    vacancy_frac removes that fraction of the sites (rounded down), chosen by
    the same generator."""
    params = params or ModelParams()
    rng = np.random.Generator(np.random.PCG64(seed))
    R = bcc_positions(ncell, a)
    n_vac = int(vacancy_frac * R.shape[0])
    if n_vac > 0:
        keep = np.sort(rng.permutation(R.shape[0])[n_vac:])
        R = R[keep]
    R = R + rng.normal(0.0, sigma, size=R.shape)
    V = maxwell_velocities(rng, R.shape[0], params.mass_amu, T_K)
    n0 = initial_n(rng, R.shape[0], m0=m0, noise=noise)
    cell = np.full(3, ncell * a)
    recipe = dict(ncell=int(ncell), seed=int(seed), sigma=float(sigma), a=float(a),
                  T_K=float(T_K), m0=float(m0), noise=float(noise),
                  vacancy_frac=float(vacancy_frac))
    return Workload(name=name, ncell=ncell, a=a, R=R, V=V, n0=n0, cell=cell,
                    params=params, steps=steps, recipe=recipe)


# The three single-GPU workloads of the hot path (16, 128 and 1024 atoms).
def fe16() -> Workload:
    """16-atom cell (2x2x2 bcc), Krylov rank 4, dt 0.5 fs, 100 steps."""
    return make_cell(2, seed=SEED_BASE + 1, name="fe16_bcc2x2x2",
                     params=ModelParams(krylov_rank=4), steps=100)


def fe128() -> Workload:
    """128-atom cell (4x4x4 bcc), ferromagnetic start, rank 6, 1000 steps."""
    return make_cell(4, seed=SEED_BASE + 2, name="fe128_bcc4x4x4",
                     params=ModelParams(krylov_rank=6), steps=1000)


def fe1024() -> Workload:
    """1024-atom cell (8x8x8 bcc, 9216 orbitals x 2 spins), rank 8, 500 steps."""
    return make_cell(8, seed=SEED_BASE + 3, name="fe1024_bcc8x8x8",
                     params=ModelParams(krylov_rank=8), steps=500)


def fe2000() -> Workload:
    """2000-atom cell (10x10x10 bcc, 18000 orbitals x 2 spins, padded to 18048
    in the mixed forms), rank 8."""
    return make_cell(10, seed=SEED_BASE + 5, name="fe2000_bcc10x10x10",
                     params=ModelParams(krylov_rank=8), steps=10000)


def replica_set(count: int = 48) -> list:
    """Uneven replicas for the batched form: bcc n x n x n cells with n in
    3..6 (54 to 432 sites), 0-5 % vacancies and displacements sigma in
    0.03-0.10 A, all drawn from one seeded generator; Krylov rank 6."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE + 4))
    out = []
    for i in range(count):
        ncell = int(rng.integers(3, 7))
        vac = float(rng.uniform(0.0, 0.05))
        sigma = float(rng.uniform(0.03, 0.10))
        out.append(make_cell(ncell, seed=SEED_BASE + 1000 + i, sigma=sigma, vacancy_frac=vac,
                             name=f"replica{i:02d}_bcc{ncell}", params=ModelParams(krylov_rank=6),
                             steps=200))
    return out


def general_model(p: ModelParams, l_resolved: bool = True) -> ModelParams:
    """The iron-like model with the paper-general features on: overlap
    integrals S0_b = -V0_b / 15 eV^-1 (overlap and hopping integrals of
    opposite sign, as usual; S stays well conditioned, eigenvalues 0.58 to
    2.29 in these bcc cells) with the hopping integrals' decay, and
    l-dependent Stoner parameters J_s = J_p = -0.1, J_d = -0.3 eV."""
    return p.replace(S0=tuple(-v / 15.0 for v in p.V0), s_decay=p.q_decay,
                     l_resolved=bool(l_resolved), J_l=(-0.1, -0.1, -0.3))


def shell_resolved_n(n_atom: np.ndarray) -> np.ndarray:
    """Per-atom extended vector [n_up; n_dn] (2 N_at) -> l-resolved layout
    [n_up (N_at x 3); n_dn (N_at x 3)] with each atom's occupation on its
    d shell (s and p shells neutral)."""
    n_atom = np.asarray(n_atom, dtype=np.float64)
    nat = n_atom.size // 2
    out = np.zeros((2, nat, 3))
    out[0, :, 2] = n_atom[:nat]
    out[1, :, 2] = n_atom[nat:]
    return out.reshape(-1)


def fe16_general() -> Workload:
    """The 16-atom cell with overlap and l-resolved charges and spins."""
    w = fe16()
    w.params = general_model(w.params)
    w.n0 = shell_resolved_n(w.n0)
    w.shell_resolved_n0 = True
    w.name = "fe16_bcc2x2x2_general"
    return w


def fe54_general() -> Workload:
    """54-atom cell (3x3x3 bcc, 486 orbitals: ragged tiles) of the general model."""
    w = make_cell(3, seed=SEED_BASE + 6, name="fe54_bcc3x3x3_general",
                  params=general_model(ModelParams(krylov_rank=4)))
    w.n0 = shell_resolved_n(w.n0)
    w.shell_resolved_n0 = True
    return w


def fe128_general() -> Workload:
    """The 128-atom cell of the general model (overlap, shells resolved)."""
    w = fe128()
    w.params = general_model(w.params)
    w.n0 = shell_resolved_n(w.n0)
    w.shell_resolved_n0 = True
    w.name = "fe128_bcc4x4x4_general"
    return w


def fe1024_general() -> Workload:
    """The 1024-atom cell of the general model (overlap, shells resolved)."""
    w = fe1024()
    w.params = general_model(w.params)
    w.n0 = shell_resolved_n(w.n0)
    w.shell_resolved_n0 = True
    w.name = "fe1024_bcc8x8x8_general"
    return w


WORKLOADS = {"fe16": fe16, "fe128": fe128, "fe1024": fe1024, "fe2000": fe2000,
             "fe16_general": fe16_general, "fe54_general": fe54_general,
             "fe128_general": fe128_general, "fe1024_general": fe1024_general}


# ---------------------------------------------------------------------------
# JSON configurations: one file per workload, holding the parameter set (the
# fields of sxl_params, one to one) and the seeded recipe of the cell.
CONFIG_VERSION = 1


def config(w: Workload, precision: Optional[str] = None) -> dict:
    """The JSON-able configuration that regenerates w exactly: parameters,
    the make_cell recipe (lattice, seeds, displacements, vacancies,
    temperature, initial moments), the step count and, optionally, the
    arithmetic form a run should use."""
    if w.recipe is None:
        raise ValueError("workload was not made by make_cell")
    params = {k: (list(v) if isinstance(v, tuple) else v)
              for k, v in dataclasses.asdict(w.params).items()}
    out = {"version": CONFIG_VERSION, "name": w.name, "lattice": "bcc",
           "cell": dict(w.recipe), "steps": int(w.steps),
           "shell_resolved_n0": bool(w.shell_resolved_n0), "params": params}
    if precision is not None:
        out["precision"] = precision
    return out


def from_config(cfg: dict) -> Workload:
    """The workload a configuration describes (inverse of config())."""
    if cfg.get("version") != CONFIG_VERSION or cfg.get("lattice", "bcc") != "bcc":
        raise ValueError("unsupported workload configuration")
    fields = {f.name for f in dataclasses.fields(ModelParams)}
    unknown = set(cfg["params"]) - fields
    if unknown:
        raise ValueError(f"unknown parameters {sorted(unknown)}")
    params = ModelParams(**{k: (tuple(v) if isinstance(v, list) else v)
                            for k, v in cfg["params"].items()})
    c = dict(cfg["cell"])
    ncell = c.pop("ncell")
    w = make_cell(ncell, params=params, name=cfg["name"], steps=int(cfg.get("steps", 0)), **c)
    if cfg.get("shell_resolved_n0"):
        w.n0 = shell_resolved_n(w.n0)
        w.shell_resolved_n0 = True
    return w


def load_config(path) -> Workload:
    import json
    with open(path) as f:
        return from_config(json.load(f))


def write_configs(directory) -> list:
    """Writes <name>.json for every named workload into directory."""
    import json
    import os
    os.makedirs(directory, exist_ok=True)
    paths = []
    for key, make in WORKLOADS.items():
        path = os.path.join(directory, f"{key}.json")
        with open(path, "w") as f:
            json.dump(config(make()), f, indent=1)
            f.write("\n")
        paths.append(path)
    return paths


def random_direction(n_atoms: int, seed: int) -> np.ndarray:
    """Seeded unit vector in R^{2 N_at} (a perturbation direction v)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(size=2 * n_atoms)
    return v / np.linalg.norm(v)


if __name__ == "__main__":
    import sys
    for p in write_configs(sys.argv[1] if len(sys.argv) > 1 else
                           __file__.rsplit("/", 1)[0] + "/configs"):
        print(p)
