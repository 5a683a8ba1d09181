"""Build and load the oracle's C part (oracle/spmm_omp.c: the OpenMP CSR
SpMM of the CPU baseline).  Test infrastructure: only the tests, the build
entry point and bench.py's cpu_baseline leg use it.  Plain gcc, in tree
(oracle/_lib/, not committed), same flags on x86 and Arm."""
import ctypes
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "spmm_omp.c")
LIB = os.path.join(HERE, "_lib", "liboracle_spmm.so")


def build(force=False):
    """Compile oracle/spmm_omp.c into oracle/_lib/liboracle_spmm.so (if the
    library is missing or older than the source, or force)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler for the oracle's SpMM")
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    tmp = LIB + ".tmp%d" % os.getpid()
    subprocess.check_call([cc, "-O2", "-fopenmp", "-shared", "-fPIC", SRC, "-o", tmp])
    os.replace(tmp, LIB)
    return LIB


def load():
    """ctypes handle of the oracle's SpMM library (built on demand)."""
    lib = ctypes.CDLL(build())
    P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.oracle_spmm.argtypes = [I64, P, P, P, I, P, P, I]
    lib.oracle_spmm.restype = None
    lib.oracle_spmm_seconds.argtypes = [I64, P, P, P, I, P, P, I, I]
    lib.oracle_spmm_seconds.restype = D
    return lib
