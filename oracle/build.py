"""Compile the C oracle (D3Q19 and D3Q27, each in FP64 and FP64-complex) with plain gcc.

Test infrastructure: the oracle is the slow, obviously correct CPU statement
of the method that the CUDA path is checked against.  ``-ffp-contract=off``
keeps every multiply and add separately rounded; OpenMP parallelises over
lattice planes only (the arithmetic per node is unchanged).
"""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_BUILD, "liboracle.so")
_handle = None


def build_oracle(force=False):
    """Compile ``liboracle.so`` (both velocity sets, real and complex twins linked together)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    flags = ["-O2", "-fPIC", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fno-fast-math"]
    objs = []
    for q in (19, 27):
        for tag, defs in (("real", []), ("cplx", ["-DORC_COMPLEX"])):
            obj = os.path.join(_BUILD, f"lbm_oracle_q{q}_{tag}.o")
            subprocess.check_call(["gcc", *flags, *defs, f"-DORC_Q={q}", "-c", _SRC, "-o", obj])
            objs.append(obj)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-shared", "-fopenmp", "-o", tmp, *objs, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def load_oracle():
    """Build if needed and return the ctypes handle of the oracle library."""
    global _handle
    if _handle is None:
        _handle = ctypes.CDLL(build_oracle())
    return _handle
