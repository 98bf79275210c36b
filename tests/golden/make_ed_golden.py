"""Writes the exact-diagonalisation reference curves stored next to this script.

Calls only the oracle (oracle.ed): thermal energy, specific heat and uniform
susceptibility per site (Eq. 12 Hamiltonian, Eq. 13 susceptibility) of the open 4x4
Heisenberg (J2 = 0) and J1-J2 (J2 = 0.5) lattices, sector by sector in M_z.
Usage: python tests/golden/make_ed_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import ed  # noqa: E402
from oracle.lattice import Lattice  # noqa: E402

BETAS = [round(x, 4) for x in np.concatenate([np.arange(0.0, 1.0, 0.04), np.arange(1.0, 10.01, 0.2)])]


def main():
    for J2, name in [(0.0, "ed_4x4_heisenberg.json"), (0.5, "ed_4x4_j1j2_0.5.json")]:
        lat = Lattice(4, 4, 1, J1=1.0, J2=J2)
        spec = ed.spectrum(lat)
        vals = ed.thermal(spec, lat.N, BETAS)
        e0 = min(float(ev.min()) for _, ev in spec)
        out = dict(lattice="4x4 open", J1=1.0, J2=J2, ground_energy_site=e0 / lat.N,
                   beta=BETAS, E_site=vals[:, 0].tolist(), C_site=vals[:, 1].tolist(),
                   chi_site=vals[:, 2].tolist(),
                   source="oracle.ed sector-blocked exact diagonalisation")
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(out, f, indent=1)
        print(name, "E0/N =", e0 / lat.N)


if __name__ == "__main__":
    main()
