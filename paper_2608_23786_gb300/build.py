"""Build libmclbm.so (D3Q19) and libmclbm_d3q27.so (D3Q27) for sm_103a with nvcc (no
CMake, no torch extension machinery).

Each translation unit under csrc/ is compiled in parallel, once per velocity set; the
shared libraries are written to _build/ inside the package so the loaded .so is in-tree.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libmclbm.so")  # D3Q19, the paper's velocity set
LIB27 = os.path.join(BUILD, "libmclbm_d3q27.so")  # the same library for D3Q27 (-DMCLBM_D3Q27)
LATTICE_LIBS = {19: LIB, 27: LIB27}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden"]


def _nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmclbm")
    return path


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _build_one(nvcc, headers, lib, objdir, defs, force, verbose, extra_flags, pool):
    os.makedirs(objdir, exist_ok=True)
    objs, jobs = [], []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, *headers]):
            jobs.append([nvcc, *ARCH, *NVCC_FLAGS, *defs, *extra_flags, "-c", src, "-o", obj])
    return lib, objs, jobs


def build(force=False, verbose=False, extra_flags=()):
    """Compile every csrc/*.cu twice (D3Q19 and D3Q27) and link _build/libmclbm.so and
    _build/libmclbm_d3q27.so; returns the D3Q19 library's path."""
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(PKG), "include", "mclbm.h"))
    nvcc = _nvcc()
    plans = [_build_one(nvcc, headers, LIB, BUILD, [], force, verbose, extra_flags, None),
             _build_one(nvcc, headers, LIB27, os.path.join(BUILD, "d3q27"), ["-DMCLBM_D3Q27"], force, verbose,
                        extra_flags, None)]
    jobs = [j for _, _, js in plans for j in js]
    workers = max(1, min(16, os.cpu_count() or 1, len(jobs)))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
            if verbose or res.returncode != 0:
                print(" ".join(cmd))
                print(res.stdout + res.stderr)
            if res.returncode != 0:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    for lib, objs, js in plans:
        if force or js or _stale(lib, objs):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
            res = subprocess.run(cmd, capture_output=True, text=True)
            if res.returncode != 0:
                print(" ".join(cmd))
                print(res.stdout + res.stderr)
                raise RuntimeError(f"linking {os.path.basename(lib)} failed")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
