"""Write ``oracle_regression.json``: outputs of the oracle on tiny seeded lattices.

The paper prints no numerical output of any operator or solver (its tables are
performance figures), so no fixture here holds a value from the paper. This
file instead freezes the oracle's own results, computed only by ``oracle/`` on
inputs from ``synthetic/``, so that a later change to the oracle's arithmetic
shows up as a failing regression test and has to be justified against the
mathematics. The values are reductions (norms, inner products, a few
components) rather than whole fields to keep the file small.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import dwf, force, wilson  # noqa: E402
from synthetic import gauge_field, gaussian_spinor  # noqa: E402

BC = (1.0, 1.0, 1.0, -1.0)
DIMS = (2, 2, 2, 4)
MASS = 0.1
M5, MF, LS = 1.8, 0.02, 4


def _cplx(z):
    return [float(np.real(z)), float(np.imag(z))]


def compute():
    U = gauge_field(DIMS, "haar", 1201)
    psi = gaussian_spinor(DIMS, 1202)
    chi = gaussian_spinor(DIMS, 1203)
    out = {}
    hp = wilson.hop(U, psi, BC)
    out["wilson_hop_norm"] = float(np.linalg.norm(hp))
    out["wilson_hop_first_site"] = [_cplx(z) for z in hp.reshape(-1)[:4]]
    out["chi_dag_D_psi"] = _cplx(np.vdot(chi, wilson.dirac(U, psi, MASS, BC)))
    pe = wilson.restrict(psi, 0)
    out["schur_dag_schur_norm"] = float(np.linalg.norm(wilson.schur_dag_schur(U, pe, MASS, BC)))
    psi5 = gaussian_spinor(DIMS, 1204, lead=(LS,))
    d5 = dwf.dirac(U, psi5, M5, MF, BC)
    out["dwf_dirac_norm"] = float(np.linalg.norm(d5))
    out["dwf_m5op_inv_norm"] = float(np.linalg.norm(dwf.m5op_inv(psi5, M5, MF)))
    S, grad, F, X, Y = force.force(U, psi, 0.05, BC, tol=1e-14)
    out["force_action"] = float(S)
    out["force_F_norm"] = float(np.linalg.norm(F))
    out["force_F_first_link_diag_real"] = [float(np.real(F.reshape(-1, 3, 3)[0][k, k])) for k in range(3)]
    return out


def main():
    data = {
        "what": "oracle outputs on tiny seeded lattices (regression fixture; not values from the paper)",
        "inputs": {"dims": list(DIMS), "bc": list(BC), "mass": MASS, "M5": M5, "mf": MF, "Ls": LS,
                   "gauge": "haar seed 1201", "psi": "gaussian seed 1202", "chi": "gaussian seed 1203",
                   "psi5": "gaussian seed 1204", "force_mass": 0.05},
        "values": compute(),
    }
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as fh:
        json.dump(data, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
