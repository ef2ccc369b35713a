"""CPU oracle for the NNQS local-energy path (arXiv 2306.16705).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline arm import this package.  The CUDA library never does, and this
package imports nothing of the CUDA path; both read their inputs from
``paper_2306_16705_gb300.inputs`` only.

Everything here is plain and slow on purpose: FP64 throughout, each function
following one passage of the paper (cited in its docstring), with library
primitives (sorting, ``numpy.linalg.eigh``, matrix products) as the only
building blocks beyond the written-out arithmetic.

Modules
  hamiltonian  Eq. (eham) -> Eq. (sham) by Jordan-Wigner operator algebra,
               Alg. 1 folding and grouping, the determinant-rule matrix used
               to pin it, exact diagonalisation, Eq. (Eloc).
  ansatz       The transformer amplitude / MLP phase of Sec. 3.1 with the
               number mask of Sec. 3.3, forward and hand-written reverse mode.
  vmc          Eq. (energy) statistics, the gradient estimator of Sec. 2.1,
               exact enumeration of p(x), the Adam and AdamW updates and the
               warm-up learning rate of Sec. 4.1.
  ladder       The CPU rungs of the local-energy speed-up ladder of Sec. 4.3
               (bare, SA+FUSE, +LUT), all computing the sample-aware sum.

Parity status: every function is pinned by a ``-m "not gpu"`` test
(``tests/test_oracle_*.py``) except where a docstring says "parity unpinned".
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "ladder.c")]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c and ladder.c with gcc (OpenMP over samples) into _build/."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                           *_SRCS, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    """The compiled oracle library (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            i64, p = ctypes.c_int64, ctypes.c_void_p
            L.oracle_jw_build.restype = i64
            L.oracle_jw_build.argtypes = [ctypes.c_int, p, p, ctypes.c_double]
            L.oracle_jw_fetch.restype = ctypes.c_int
            L.oracle_jw_fetch.argtypes = [p, p, p, p]
            L.oracle_coupled.restype = i64
            L.oracle_coupled.argtypes = [ctypes.c_int, i64, p, p, p, p, ctypes.c_int,
                                         ctypes.c_int, p, p, i64]
            L.oracle_eloc_lut.restype = ctypes.c_int
            L.oracle_eloc_lut.argtypes = [ctypes.c_int, i64, p, p, p, i64, p, p, i64, p,
                                          ctypes.c_int, ctypes.c_int, p]
            L.ladder_eloc.restype = ctypes.c_int
            L.ladder_eloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, p, p, p, p, i64, p, p,
                                      p, p, i64, p, p]
            _lib = L
    return _lib
