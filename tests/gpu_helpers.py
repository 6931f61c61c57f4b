"""Shared helpers of the GPU parity tests (library <-> oracle mapping)."""
import numpy as np

import oracle
from paper_2608_23786_gb300 import mclbm


def lib_to_oracle_perm(lattice=19):
    """perm[i] = oracle index of the library's velocity i (matched by the velocity vector)."""
    c_lib, _ = mclbm.mclbm_lattice(lattice)
    c_orc, _, _ = oracle.lattice(lattice)
    return np.array([int(np.where((c_orc == c_lib[i]).all(1))[0][0]) for i in range(lattice)])


def lib_populations(ens):
    """All samples' pre-collision populations in the oracle's velocity order, [M][Q][N][N][N]."""
    q = getattr(ens, "lattice", 19)
    perm = lib_to_oracle_perm(q)
    inv = np.argsort(perm)
    out = np.empty((ens.M, q, ens.N, ens.N, ens.N))
    for m in range(ens.M):
        f = ens.populations(m).cpu().numpy()
        out[m] = f[inv]
    return out


def oracle_to_lib(f_orc):
    """One sample's populations from oracle order to library order."""
    return f_orc[lib_to_oracle_perm(len(f_orc))]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
