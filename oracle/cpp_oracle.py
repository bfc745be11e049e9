"""ctypes wrapper of the plain FP64 C++ oracle (oracle/cpp/roks_oracle.cpp).

TEST INFRASTRUCTURE, like the rest of this package: only tests/,
__graft_entry__.smoke() and bench.py's CPU-baseline legs may load it.  It is
built with the host compiler (g++ -O3 -fopenmp; no architecture flags, so the
same source builds on x86 and Arm hosts) into oracle/cpp/ on first use.

CppSystem mirrors the parts of oracle.roks.System that the band apply needs:
the basis, the class densities, the potentials with their energies, and F,
S of a set of bands (threads over bands)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpp", "roks_oracle.cpp")
LIB = os.path.join(HERE, "cpp", "libroks_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp"
        subprocess.run(["g++", "-O3", "-fcx-limited-range", "-fopenmp", "-fPIC", "-shared", "-std=c++17", "-o", tmp, SRC],
                       check=True)
        os.replace(tmp, LIB)
    return LIB


def load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        lib.ro_create.restype = P
        lib.ro_create.argtypes = [C.c_double, C.c_int, C.c_double, C.c_int, C.c_int, C.c_double, C.c_int, dp, ip,
                                  dp, dp, ip, ip, ip, dp, dp, dp]
        lib.ro_destroy.argtypes = [P]
        for f in ("ro_npw", "ro_nproj"):
            getattr(lib, f).restype = C.c_int
            getattr(lib, f).argtypes = [P]
        lib.ro_miller.restype = C.POINTER(C.c_int32)
        lib.ro_miller.argtypes = [P]
        lib.ro_vloc.restype = dp
        lib.ro_vloc.argtypes = [P]
        lib.ro_projectors.restype = dp
        lib.ro_projectors.argtypes = [P]
        lib.ro_densities.argtypes = [P, dp, C.c_int64, C.c_int, C.c_int, dp, C.c_int]
        lib.ro_potentials.argtypes = [P, dp, dp, dp]
        lib.ro_apply.argtypes = [P, dp, C.c_int64, C.c_int, ip, dp, dp, dp, C.c_int]
        _lib = lib
    return _lib


def _d(a):
    """Pointer to the first double of an array (a complex array's re, im pairs)."""
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class CppSystem:
    """One model system in the C++ oracle (see oracle.roks.System for the model)."""

    def __init__(self, cfg: dict, threads: int = 0):
        # the C++ oracle restates the Slater-exchange model without empty
        # bands (the baseline's workloads); the rest stays in oracle.roks
        if int(cfg.get("n_empty", 0)) or cfg.get("xc", "slater") != "slater":
            raise ValueError("the C++ oracle takes occupied bands and Slater exchange only")
        lib = load()
        self.cfg = cfg
        self.N = int(cfg["grid"])
        self.threads = int(threads)
        self.mode = int(cfg["mode"])
        self.n_closed = int(cfg["n_closed"])
        self.nb = self.n_closed + (0 if self.mode == 0 else 2)
        self.cls = np.array([0] * self.n_closed + list(range(1, self.nb - self.n_closed + 1)), dtype=np.int32)
        atoms = cfg["atoms"]
        pos = np.ascontiguousarray([a["pos"] for a in atoms], dtype=np.float64).reshape(-1)
        spec = np.ascontiguousarray([a["species"] for a in atoms], dtype=np.int32)
        depth = np.ascontiguousarray([a["depth"] for a in atoms], dtype=np.float64)
        width = np.ascontiguousarray([a["width"] for a in atoms], dtype=np.float64)
        sps = cfg["species"]
        nproj = np.ascontiguousarray([len(sp["l"]) for sp in sps], dtype=np.int32)
        l = np.ascontiguousarray(np.concatenate([np.asarray(sp["l"], dtype=np.int32) for sp in sps]), dtype=np.int32)
        m = np.ascontiguousarray(np.concatenate([np.asarray(sp["m"], dtype=np.int32) for sp in sps]), dtype=np.int32)
        rc = np.ascontiguousarray(np.concatenate([np.asarray(sp["rc"], dtype=np.float64) for sp in sps]))
        D = np.ascontiguousarray(np.concatenate([np.asarray(sp["D"], dtype=np.float64).reshape(-1) for sp in sps]))
        Q = np.ascontiguousarray(np.concatenate([np.asarray(sp["Q"], dtype=np.float64).reshape(-1) for sp in sps]))
        self._keep = (pos, spec, depth, width, nproj, l, m, rc, D, Q)
        self.h = lib.ro_create(float(cfg["L"]), self.N, float(cfg["ecut"]), self.mode, self.n_closed,
                               float(cfg.get("alpha", 0.0)), len(atoms), _d(pos), _i(spec), _d(depth), _d(width),
                               _i(nproj), _i(l), _i(m), _d(rc), _d(D), _d(Q))
        if not self.h:
            raise ValueError("grid too small for the sphere")
        self.npw = lib.ro_npw(self.h)
        self.nproj = lib.ro_nproj(self.h)
        self.miller = np.ctypeslib.as_array(lib.ro_miller(self.h), shape=(self.npw, 3)).astype(np.int64)

    def close(self):
        if self.h:
            load().ro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vloc(self) -> np.ndarray:
        return np.ctypeslib.as_array(load().ro_vloc(self.h), shape=(self.N ** 3,)).copy()

    def projectors(self) -> np.ndarray:
        a = np.ctypeslib.as_array(load().ro_projectors(self.h), shape=(self.nproj * self.npw * 2,))
        return (a[0::2] + 1j * a[1::2]).reshape(self.nproj, self.npw).T.copy()

    def class_densities(self, Psi: np.ndarray, b0: int = 0) -> np.ndarray:
        """rho_k(r) of the columns of Psi (bands b0 ...), shape (3, N^3)."""
        X = np.asfortranarray(Psi, dtype=np.complex128)
        rho = np.zeros(3 * self.N ** 3)
        load().ro_densities(self.h, _d(X), X.shape[0], b0, X.shape[1], _d(rho), self.threads)
        return rho.reshape(3, -1)

    def potentials(self, rho3: np.ndarray):
        """(Vk (3, N^3), energies {H, x_M, x_T, loc})."""
        r = np.ascontiguousarray(rho3, dtype=np.float64).reshape(-1)
        Vk = np.zeros(3 * self.N ** 3)
        E = np.zeros(4)
        load().ro_potentials(self.h, _d(r), _d(Vk), _d(E))
        return Vk.reshape(3, -1), dict(zip(("H", "x_M", "x_T", "loc"), E.tolist()))

    def apply(self, Psi: np.ndarray, Vk: np.ndarray, classes=None, want_s: bool = True):
        """F^k|n> and S|n> of the columns of Psi (classes: one per column)."""
        X = np.asfortranarray(Psi, dtype=np.complex128)
        cls = np.ascontiguousarray(self.cls if classes is None else classes, dtype=np.int32)
        F = np.zeros_like(X, order="F")
        S = np.zeros_like(X, order="F") if want_s else None
        V = np.ascontiguousarray(Vk, dtype=np.float64).reshape(-1)
        load().ro_apply(self.h, _d(X), X.shape[0], X.shape[1], _i(cls), _d(V),
                        _d(F), _d(S) if S is not None else None, self.threads)
        return F, S
