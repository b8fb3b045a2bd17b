"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

The oracle is plain C++ (``mr_oracle.cpp``) compiled with
``-O2 -ffp-contract=off``; it shares no code with the CUDA library.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mr_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")


def build_oracle(force=False):
    """Compile liboracle.so next to the source (rebuilds when the source is newer)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared",
           "-o", tmp, _SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class OracleParams(C.Structure):
    _fields_ = [("dim", C.c_int32), ("Bs", C.c_int32), ("ng", C.c_int32),
                ("nvar", C.c_int32), ("Jmin", C.c_int32), ("Jmax", C.c_int32),
                ("rhs_kind", C.c_int32), ("ic_kind", C.c_int32),
                ("norm_kind", C.c_int32), ("max_rounds", C.c_int32),
                ("L", C.c_double), ("eps", C.c_double),
                ("x0", C.c_double * 3), ("rhs", C.c_double * 8),
                ("ic", C.c_double * 32)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build_oracle())
        vp = C.c_void_p
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [C.POINTER(OracleParams)]
        for name in ("orc_destroy", "orc_init_tree", "orc_sync", "orc_details", "orc_filter"):
            getattr(lib, name).argtypes = [vp]
            getattr(lib, name).restype = None
        lib.orc_nblocks.argtypes = [vp]; lib.orc_nblocks.restype = C.c_int64
        lib.orc_errors.argtypes = [vp]; lib.orc_errors.restype = C.c_int64
        lib.orc_refine.argtypes = [vp, C.c_int]; lib.orc_refine.restype = None
        lib.orc_rk4.argtypes = [vp, C.c_double, C.c_double]; lib.orc_rk4.restype = None
        lib.orc_step.argtypes = [vp, C.c_double, C.c_double]; lib.orc_step.restype = None
        lib.orc_flags.argtypes = [vp, C.c_uint64]; lib.orc_flags.restype = C.c_int
        lib.orc_coarsen.argtypes = [vp]; lib.orc_coarsen.restype = C.c_int
        lib.orc_coarsen_until_stable.argtypes = [vp]
        lib.orc_coarsen_until_stable.restype = C.c_int
        lib.orc_nrel.argtypes = [vp]; lib.orc_nrel.restype = C.c_int
        lib.orc_hilbert.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int64)]
        lib.orc_hilbert.restype = C.c_uint64
        lib.orc_get_blocks.argtypes = [vp] + [C.c_void_p] * 7
        lib.orc_get_blocks.restype = None
        lib.orc_get_tiles.argtypes = [vp, C.c_void_p]; lib.orc_get_tiles.restype = None
        lib.orc_set_blocks.argtypes = [vp, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]
        lib.orc_set_blocks.restype = None
        lib.orc_set_ic.argtypes = [vp, C.c_double]; lib.orc_set_ic.restype = None
        lib.orc_neighbors.argtypes = [vp, C.c_void_p, C.c_void_p]
        lib.orc_neighbors.restype = None
        lib.orc_rhs.argtypes = [vp, C.c_double, C.c_void_p]; lib.orc_rhs.restype = None
        lib.orc_error.argtypes = [vp, C.c_double, C.c_void_p]; lib.orc_error.restype = None
        lib.orc_set_flags.argtypes = [vp, C.c_void_p]; lib.orc_set_flags.restype = None
        lib.orc_set_mdet.argtypes = [vp, C.c_void_p]; lib.orc_set_mdet.restype = None
        lib.orc_close_refine.argtypes = [vp]; lib.orc_close_refine.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One tree of the FP64 oracle.  ``cfg`` is a dict with the OracleParams fields."""

    RHS = {"adv": 0, "swirl": 1, "ns": 2, "ns_skew": 3}
    IC = {"gauss": 0, "mixing": 1, "none": 2, "shear_layer": 3}

    def __init__(self, cfg):
        lib = _load()
        p = OracleParams()
        p.dim = cfg["dim"]; p.Bs = cfg.get("Bs", 17); p.ng = cfg.get("ng", 4)
        p.nvar = cfg.get("nvar", 1); p.Jmin = cfg["Jmin"]; p.Jmax = cfg["Jmax"]
        p.rhs_kind = self.RHS[cfg.get("rhs", "adv")]
        p.ic_kind = self.IC[cfg.get("ic", "gauss")]
        p.norm_kind = cfg.get("norm_kind", 0)
        p.max_rounds = cfg.get("max_rounds", 0)
        p.L = cfg.get("L", 1.0); p.eps = cfg.get("eps", 1e-3)
        for a, v in enumerate(cfg.get("x0", (0.0, 0.0, 0.0))):
            p.x0[a] = v
        for a, v in enumerate(cfg.get("rhs_params", ())):
            p.rhs[a] = v
        for a, v in enumerate(cfg.get("ic_params", ())):
            p.ic[a] = v
        self.p = p
        self.lib = lib
        self.h = lib.orc_create(C.byref(p))
        self.dim, self.B, self.g, self.nvar = p.dim, p.Bs, p.ng, p.nvar

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    # --- method steps -----------------------------------------------------
    def init_tree(self):
        self.lib.orc_init_tree(self.h)

    def sync(self):
        self.lib.orc_sync(self.h)

    def refine(self, mode=0):
        self.lib.orc_refine(self.h, mode)

    def rk4(self, t, dt):
        self.lib.orc_rk4(self.h, t, dt)

    def details(self):
        self.lib.orc_details(self.h)

    def filter(self):
        """Shock-capturing filter of a Navier-Stokes state (Sec. 4); no-op unless r_th > 0."""
        self.lib.orc_filter(self.h)

    def flags(self, seed=0):
        return self.lib.orc_flags(self.h, seed)

    def coarsen(self):
        return self.lib.orc_coarsen(self.h)

    def coarsen_until_stable(self):
        return self.lib.orc_coarsen_until_stable(self.h)

    def step(self, t, dt):
        self.lib.orc_step(self.h, t, dt)

    def close_refine(self):
        """Gradedness closure of the +1 statuses (Sec. 2.2, 2.3); returns the number raised."""
        return self.lib.orc_close_refine(self.h)

    def set_flags(self, flags):
        """Refinement statuses in Hilbert (export) order."""
        f = np.ascontiguousarray(flags, np.int8)
        assert len(f) == self.n
        self.lib.orc_set_flags(self.h, _ptr(f))

    def set_mdet(self, mdet):
        """Largest block details in Hilbert (export) order."""
        m = np.ascontiguousarray(mdet, np.float64)
        assert len(m) == self.n
        self.lib.orc_set_mdet(self.h, _ptr(m))

    def set_ic(self, t=0.0):
        self.lib.orc_set_ic(self.h, t)

    # --- inspection -------------------------------------------------------
    @property
    def n(self):
        return int(self.lib.orc_nblocks(self.h))

    @property
    def errors(self):
        return int(self.lib.orc_errors(self.h))

    @property
    def nrel(self):
        return int(self.lib.orc_nrel(self.h))

    def npts(self):
        return self.B ** self.dim

    def blocks(self, fields=True):
        n = self.n
        out = dict(level=np.zeros(n, np.int32), coords=np.zeros((n, 3), np.int64),
                   treecode=np.zeros(n, np.uint64), hkey=np.zeros(n, np.uint64),
                   flag=np.zeros(n, np.int8), mdet=np.zeros(n, np.float64))
        f = np.zeros((n, self.nvar) + (self.B,) * self.dim, np.float64) if fields else None
        self.lib.orc_get_blocks(self.h, _ptr(out["level"]), _ptr(out["coords"]),
                                _ptr(out["treecode"]), _ptr(out["hkey"]), _ptr(out["flag"]),
                                _ptr(out["mdet"]), _ptr(f))
        out["fields"] = f
        return out

    def tiles(self):
        T = self.B + 2 * self.g
        t = np.zeros((self.n, self.nvar) + (T,) * self.dim, np.float64)
        self.lib.orc_get_tiles(self.h, _ptr(t))
        return t

    def set_blocks(self, level, coords, fields=None):
        level = np.ascontiguousarray(level, np.int32)
        coords = np.ascontiguousarray(coords, np.int64).reshape(-1, 3)
        if fields is not None:
            fields = np.ascontiguousarray(fields, np.float64)
        self.lib.orc_set_blocks(self.h, len(level), _ptr(level), _ptr(coords), _ptr(fields))

    def neighbors(self):
        n, R = self.n, self.nrel
        nbr = np.zeros((n, R), np.int32)
        dl = np.zeros((n, R), np.int8)
        self.lib.orc_neighbors(self.h, _ptr(nbr), _ptr(dl))
        return nbr, dl

    def rhs(self, t=0.0):
        out = np.zeros((self.n, self.nvar) + (self.B,) * self.dim, np.float64)
        self.lib.orc_rhs(self.h, t, _ptr(out))
        return out

    def error(self, t):
        out = np.zeros(4, np.float64)
        self.lib.orc_error(self.h, t, _ptr(out))
        return dict(l2=out[0] / out[1], linf=out[2] / out[3], l2_abs=out[0], linf_abs=out[2])

    @staticmethod
    def hilbert(dim, bits, cell):
        c = (C.c_int64 * 3)(*[int(x) for x in (list(cell) + [0, 0, 0])[:3]])
        return int(_load().orc_hilbert(dim, bits, c))
