"""Shared helpers of the GPU parity tests (library <-> oracle mapping)."""
import numpy as np

import oracle
from paper_2608_23786_gb300 import mclbm


def lib_to_oracle_perm():
    """perm[i] = oracle index of the library's velocity i (matched by the velocity vector)."""
    c_lib, _ = mclbm.mclbm_lattice()
    c_orc, _, _ = oracle.lattice()
    return np.array([int(np.where((c_orc == c_lib[i]).all(1))[0][0]) for i in range(19)])


def lib_populations(ens):
    """All samples' pre-collision populations in the oracle's velocity order, [M][19][N][N][N]."""
    perm = lib_to_oracle_perm()
    inv = np.argsort(perm)
    out = np.empty((ens.M, 19, ens.N, ens.N, ens.N))
    for m in range(ens.M):
        f = ens.populations(m).cpu().numpy()
        out[m] = f[inv]
    return out


def oracle_to_lib(f_orc):
    """One sample's populations from oracle order to library order."""
    return f_orc[lib_to_oracle_perm()]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
