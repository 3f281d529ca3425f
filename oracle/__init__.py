"""FP64 CPU oracle for spin-polarized XL-BOMD (arXiv 2303.03529).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this package.  The
product path (the CUDA library and its Python binding) never imports it and
fails loudly when its extension is missing.

The oracle is plain, slow and written to be checked against the paper by eye:
  * model.py     Slater-Koster H0 (image-summed), screened Coulomb gamma,
                 spin-resolved Hamiltonians H_sigma[n]      (Sec. III.A)
  * electronic.py  D_sigma = f_FD(H_sigma) by dense eigendecomposition with
                 one common chemical potential, Mulliken q and m, first-order
                 response q_v by eigenbasis divided differences (Eqs. D_min,
                 fv), Jacobian columns                       (Secs. II.C, II.G)
  * kernel.py    preconditioned low-rank Krylov kernel       (Eq. mIJacobian)
  * energy.py    shadow energy and forces at constant n     (Eqs. ShadowELatte,
                 EqMot)
  * dynamics.py  modified Verlet with dissipation, XL-BOMD loop, SCF with the
                 kernel quasi-Newton mixer                   (Eqs. Integration, QN)

It shares no code with the CUDA path.  Inputs come from
paper_2303_03529_gb300.workload (seeded generators only) or from the caller.
Parameters are read by attribute from any object with the fields of
workload.ModelParams.
"""
