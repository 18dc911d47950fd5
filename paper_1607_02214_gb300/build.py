"""Build the in-tree CUDA library libppmlr_gb300.so for sm_103a.

Each translation unit is compiled in parallel with one -gencode target; the
objects are linked with nvcc into a shared library next to this file.  The exact
FP64 sweep and CFL units and the host units are compiled without
floating-point contraction (-fmad=false, -ffp-contract=off); the default FP64
units use contraction; the mixed-precision units use contraction and fast
FP32 division/square root.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libppmlr_gb300.so")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                 "-I", os.path.join(HERE, "..", "include")]
UNITS = {
    "api.cu": ["-fmad=false"],
    "ensemble.cu": ["-fmad=false"],
    "cfl.cu": ["-fmad=false"],
    "cfl_fp64.cu": ["-fmad=true"],
    "cfl_noalloc.cu": ["-fmad=false"],
    "sweep_fp64.cu": ["-fmad=true"],
    "sweep_fp64_exact.cu": ["-fmad=false"],
    "sweep_mixed.cu": ["-fmad=true", "-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
    "cfl_mixed.cu": ["-fmad=true", "-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
    "ionosphere.cu": ["-fmad=true"],
    "selftest.cu": ["-fmad=true"],
    "pipe_rate.cu": ["-fmad=true"],
}


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))] + \
        [os.path.join(HERE, "..", "include", "ppmlr.h")]


# bounds-checked build (-DPPMLR_CHECK): every kernel index of the sweeps is
# tested against its array; for the tests, not for timing
LIB_CHECK = os.path.join(HERE, "libppmlr_gb300_check.so")
OUT_CHECK = os.path.join(HERE, "_build_check")


def up_to_date(lib=LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _compile(unit, verbose, check=False):
    src = os.path.join(CSRC, unit)
    obj = os.path.join(OUT_CHECK if check else OUT, unit.replace(".cu", ".o"))
    cmd = [NVCC, *COMMON, *UNITS[unit], *(["-DPPMLR_CHECK"] if check else []), "-c", src, "-o", obj]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {unit}:\n{r.stderr}")
    return obj, r.stderr


def build(force: bool = False, verbose: bool = False, check: bool = False) -> str:
    """Build the library (check=True: the bounds-checked variant, a separate
    file); returns its path."""
    lib = LIB_CHECK if check else LIB
    if not force and up_to_date(lib):
        return lib
    os.makedirs(OUT_CHECK if check else OUT, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(lambda u: _compile(u, verbose, check), UNITS))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, check="--check" in sys.argv))
