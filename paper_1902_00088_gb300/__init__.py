"""GB300 block-based multiresolution solver (Sroka et al., arXiv:1902.00088).

Thin ctypes binding of the C ABI in ``include/mr.h``.  Every function here only
marshals arguments; all computation runs in the CUDA kernels of
``_build/libmr.so``.  There is no CPU fallback: if the library is missing the
import of the binding raises.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmr.so")

MR_OK, MR_EINVAL, MR_ENOMEM, MR_ECAPACITY, MR_ECUDA, MR_ETIMEOUT, MR_ENAN, MR_EINTERNAL = range(8)
PREC = {"fp64": 0, "fp32": 1, "fp32_acc64": 2}
RHS = {"adv": 0, "swirl": 1, "ns": 2, "ns_skew": 3}
IC = {"gauss": 0, "mixing": 1, "none": 2, "shear_layer": 3}
ADAPT = {"refine_all": 0, "refine_flagged": 1, "coarsen": 2, "flags_only": 3, "propose": 4,
         "refine_step": 5}
STATUS = {0: "MR_OK", 1: "MR_EINVAL", 2: "MR_ENOMEM", 3: "MR_ECAPACITY", 4: "MR_ECUDA",
          5: "MR_ETIMEOUT", 6: "MR_ENAN", 7: "MR_EINTERNAL"}


class MRError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("Bs", C.c_int32), ("ng", C.c_int32), ("nvar", C.c_int32),
                ("precision", C.c_int32), ("detail_fp64", C.c_int32), ("rhs_kind", C.c_int32),
                ("ntrees", C.c_int32), ("capacity", C.c_int64), ("max_rounds", C.c_int32),
                ("norm_kind", C.c_int32), ("L", C.c_double), ("stream", C.c_void_p)]


class TreeDesc(C.Structure):
    _fields_ = [("Jmin", C.c_int32), ("Jmax", C.c_int32), ("eps", C.c_double),
                ("x0", C.c_double * 3), ("ic_kind", C.c_int32), ("ic", C.c_double * 32),
                ("rhs", C.c_double * 8)]


class BlockInfo(C.Structure):
    _fields_ = [("level", C.c_int32), ("tree", C.c_int32), ("treecode", C.c_uint64),
                ("coords", C.c_int32 * 3), ("pad", C.c_int32), ("hilbert_key", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("ms", C.c_double * 6), ("phase_calls", C.c_int64 * 6),
                ("stage_launches", C.c_int64), ("stage_blocks", C.c_int64), ("steps", C.c_int64),
                ("det_launches", C.c_int64), ("det_blocks", C.c_int64)]


PHASES = ("refine", "stage", "details", "flags_merge", "sync_export", "filter")

BLOCK_INFO_DTYPE = np.dtype([("level", np.int32), ("tree", np.int32), ("treecode", np.uint64),
                             ("coords", np.int32, 3), ("pad", np.int32),
                             ("hilbert_key", np.uint64)])

# Exported symbols of include/mr.h: name -> (restype, argtypes)
_vp, _i32, _i64, _dp = C.c_void_p, C.c_int32, C.c_int64, C.c_void_p
SIGNATURES = {
    "mr_create": (_i32, [C.POINTER(Params), C.POINTER(TreeDesc), C.POINTER(C.c_void_p)]),
    "mr_destroy": (None, [_vp]),
    "mr_last_error": (C.c_char_p, [_vp]),
    "mr_init_tree": (_i32, [_vp]),
    "mr_set_rhs": (_i32, [_vp, _i32, _i32, _dp]),
    "mr_sync_ghosts": (_i32, [_vp]),
    "mr_filter": (_i32, [_vp]),
    "mr_rk_step": (_i32, [_vp, _dp, _dp]),
    "mr_adapt": (_i32, [_vp, _i32]),
    "mr_step": (_i32, [_vp, _dp, _dp]),
    "mr_num_blocks": (_i32, [_vp, _i32, C.POINTER(C.c_int64)]),
    "mr_get_blocks": (_i32, [_vp, _i32, _i64, C.POINTER(C.c_int64), _vp, _dp]),
    "mr_get_tiles": (_i32, [_vp, _i32, _i64, C.POINTER(C.c_int64), _dp]),
    "mr_get_neighbors": (_i32, [_vp, _i32, _i64, _vp, _vp]),
    "mr_num_relations": (_i32, [_i32]),
    "mr_get_flags": (_i32, [_vp, _i32, _i64, _vp, _dp]),
    "mr_set_blocks": (_i32, [_vp, _i64, _vp, _vp, _vp, _dp]),
    "mr_set_refine_mask": (_i32, [_vp, _i64, _vp]),
    "mr_error": (_i32, [_vp, _i32, C.c_double, _dp]),
    "mr_error_noalloc": (_i32, [_vp, _i32, C.c_double, _dp]),
    "mr_launch_count": (_i64, [_vp]),
    "mr_enable_timing": (_i32, [_vp, _i32]),
    "mr_set_time": (_i32, [_vp, _dp, _dp]),
    "mr_get_time": (_i32, [_vp, _dp]),
    "mr_step_graph": (_i32, [_vp, _i64]),
    "mr_graph_mode": (_i32, [_vp]),
    "mr_set_launch_overlap": (_i32, [_vp, _i32]),
    "mr_get_launch_overlap": (_i32, [_vp]),
    "mr_get_step_history": (_i32, [_vp, _i64, _vp, C.POINTER(C.c_int64), _i32]),
    "mr_autotune": (_i32, [_vp, _i32, C.POINTER(C.c_int32)]),
    "mr_set_tuning": (_i32, [_vp, _i32, _i32]),
    "mr_set_warp_form": (_i32, [_vp, _i32, _i32]),
    "mr_set_refine_mode": (_i32, [_vp, _i32]),
    "mr_proposal_collect": (_i32, [_vp, _i32, _i64]),
    "mr_proposal_dataset": (_i32, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "mr_proposal_train": (_i32, [_vp, _vp, _i32, _i32, C.c_float, C.c_float, C.c_float, C.c_float,
                                 C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "mr_proposal_set": (_i32, [_vp, _vp, C.c_float]),
    "mr_proposal_get": (_i32, [_vp, _vp, C.POINTER(C.c_float)]),
    "mr_proposal_stats": (_i32, [_vp, _vp, _i32]),
    "mr_cnn_eval": (_i32, [_vp, _vp, _vp, _vp, _i64, C.c_float, _vp, _vp, C.POINTER(C.c_float)]),
    "mr_get_stats": (_i32, [_vp, C.POINTER(Stats)]),
    "mr_reset_stats": (_i32, [_vp]),
}

_lib = None


def load_library(path=LIB_PATH):
    """Loads libmr.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libmr.so not built: run __graft_entry__.build() or "
                              "python paper_1902_00088_gb300/build.py")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Forest:
    """A context of the C library: ``ntrees`` trees advanced together.

    Method names follow the C ABI (init_tree, set_rhs, sync_ghosts, rk_step,
    adapt, step, get_blocks, ...).
    """

    def __init__(self, dim=2, Bs=17, ng=4, nvar=1, precision="fp64", detail_fp64=False,
                 rhs="adv", trees=(), capacity=1 << 16, max_rounds=0, norm_kind=0, L=1.0,
                 stream=None):
        self.lib = load_library()
        p = Params()
        p.dim, p.Bs, p.ng, p.nvar = dim, Bs, ng, nvar
        p.precision = PREC[precision] if isinstance(precision, str) else precision
        p.detail_fp64 = int(bool(detail_fp64))
        p.rhs_kind = RHS[rhs] if isinstance(rhs, str) else rhs
        p.ntrees = len(trees)
        p.capacity = capacity
        p.max_rounds = max_rounds
        p.norm_kind = norm_kind
        p.L = L
        p.stream = stream
        arr = (TreeDesc * len(trees))()
        for k, t in enumerate(trees):
            d = arr[k]
            d.Jmin, d.Jmax, d.eps = t["Jmin"], t["Jmax"], t.get("eps", 1e-3)
            for a, v in enumerate(t.get("x0", (0.0, 0.0, 0.0))):
                d.x0[a] = v
            ic = t.get("ic", "gauss")
            d.ic_kind = IC[ic] if isinstance(ic, str) else ic
            for a, v in enumerate(t.get("ic_params", ())):
                d.ic[a] = v
            for a, v in enumerate(t.get("rhs_params", ())):
                d.rhs[a] = v
        h = C.c_void_p()
        st = self.lib.mr_create(C.byref(p), arr, C.byref(h))
        if st != MR_OK:
            raise MRError(st, "mr_create failed (invalid parameters or no device)")
        self.h = h
        self.p = p
        self.dim, self.B, self.g, self.nvar, self.ntrees = dim, Bs, ng, nvar, len(trees)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        if st != MR_OK:
            raise MRError(st, self.lib.mr_last_error(self.h).decode())

    # ---------------------------------------------------------------- steps --
    def init_tree(self):
        self._ck(self.lib.mr_init_tree(self.h))

    def set_rhs(self, rhs, params, tree=-1):
        a = np.zeros(8, np.float64)
        a[:len(params)] = params
        self._ck(self.lib.mr_set_rhs(self.h, RHS[rhs] if isinstance(rhs, str) else rhs, tree, _ptr(a)))

    def sync_ghosts(self):
        self._ck(self.lib.mr_sync_ghosts(self.h))

    def filter(self):
        """Shock-capturing filter of the Navier-Stokes state (trees with r_th > 0)."""
        self._ck(self.lib.mr_filter(self.h))

    def _td(self, t, dt):
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(t, np.float64), (self.ntrees,)))
        dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, np.float64), (self.ntrees,)))
        return t, dt

    def rk_step(self, t, dt):
        t, dt = self._td(t, dt)
        self._ck(self.lib.mr_rk_step(self.h, _ptr(t), _ptr(dt)))

    def adapt(self, mode):
        self._ck(self.lib.mr_adapt(self.h, ADAPT[mode] if isinstance(mode, str) else mode))

    def step(self, t, dt):
        t, dt = self._td(t, dt)
        self._ck(self.lib.mr_step(self.h, _ptr(t), _ptr(dt)))

    # ----------------------------------------------------------- inspection --
    def num_blocks(self, tree=-1):
        n = C.c_int64()
        self._ck(self.lib.mr_num_blocks(self.h, tree, C.byref(n)))
        return n.value

    def get_blocks(self, tree=-1, fields=True, out=None):
        """Blocks in canonical order: (info, fields).  out = (info_buf, fields_buf) writes into caller
        buffers (e.g. pinned host memory) of room for the blocks and returns views of their first n
        entries (MR_EINVAL if they are too small)."""
        if out is not None:
            ib, fb = out
            n = C.c_int64()
            self._ck(self.lib.mr_get_blocks(self.h, tree, len(ib), C.byref(n), _ptr(ib),
                                            _ptr(fb) if fields else None))
            return ib[:n.value], (fb[:n.value] if fields else None)
        n0 = self.num_blocks(tree)
        info = np.zeros(n0, BLOCK_INFO_DTYPE)
        f = np.zeros((n0, self.nvar) + (self.B,) * self.dim, np.float64) if fields else None
        n = C.c_int64()
        self._ck(self.lib.mr_get_blocks(self.h, tree, n0, C.byref(n), _ptr(info), _ptr(f)))
        return info, f

    def get_tiles(self, tree=-1):
        n0 = self.num_blocks(tree)
        T = self.B + 2 * self.g
        t = np.zeros((n0, self.nvar) + (T,) * self.dim, np.float64)
        n = C.c_int64()
        self._ck(self.lib.mr_get_tiles(self.h, tree, n0, C.byref(n), _ptr(t)))
        return t

    def get_neighbors(self, tree=-1):
        n0 = self.num_blocks(tree)
        R = self.lib.mr_num_relations(self.dim)
        nbr = np.zeros((n0, R), np.int32)
        dl = np.zeros((n0, R), np.int8)
        self._ck(self.lib.mr_get_neighbors(self.h, tree, n0, _ptr(nbr), _ptr(dl)))
        return nbr, dl

    def get_flags(self, tree=-1):
        n0 = self.num_blocks(tree)
        f = np.zeros(n0, np.int8)
        m = np.zeros(n0, np.float64)
        self._ck(self.lib.mr_get_flags(self.h, tree, n0, _ptr(f), _ptr(m)))
        return f, m

    def set_blocks(self, level, coords, fields=None, tree=None):
        level = np.ascontiguousarray(level, np.int32)
        coords = np.ascontiguousarray(np.asarray(coords).reshape(-1, 3), np.int32)
        tr = None if tree is None else np.ascontiguousarray(tree, np.int32)
        fl = None if fields is None else np.ascontiguousarray(fields, np.float64)
        self._ck(self.lib.mr_set_blocks(self.h, len(level), _ptr(level), _ptr(tr), _ptr(coords), _ptr(fl)))

    def set_refine_mask(self, mask):
        mask = np.ascontiguousarray(mask, np.int8)
        self._ck(self.lib.mr_set_refine_mask(self.h, len(mask), _ptr(mask)))

    def error(self, tree, t):
        out = np.zeros(4, np.float64)
        self._ck(self.lib.mr_error(self.h, tree, t, _ptr(out)))
        return dict(l2=out[0] / out[1], linf=out[2] / out[3], l2_abs=out[0], linf_abs=out[2])

    def error_noalloc(self, tree, t):
        """mr_error without device allocation (scratch in a static device array)."""
        out = np.zeros(4, np.float64)
        self._ck(self.lib.mr_error_noalloc(self.h, tree, t, _ptr(out)))
        return out

    def launch_count(self):
        return int(self.lib.mr_launch_count(self.h))

    def set_time(self, t, dt):
        t, dt = self._td(t, dt)
        self._ck(self.lib.mr_set_time(self.h, _ptr(t), _ptr(dt)))

    def get_time(self):
        t = np.zeros(self.ntrees, np.float64)
        self._ck(self.lib.mr_get_time(self.h, _ptr(t)))
        return t

    def step_graph(self, nsteps=1):
        self._ck(self.lib.mr_step_graph(self.h, nsteps))

    def graph_mode(self):
        return {1: "while-node", 0: "fixed-rounds", -1: None}[int(self.lib.mr_graph_mode(self.h))]

    def set_launch_overlap(self, on):
        self._ck(self.lib.mr_set_launch_overlap(self.h, 1 if on else 0))

    def launch_overlap(self):
        return bool(self.lib.mr_get_launch_overlap(self.h))

    def step_history(self, reset=True):
        n = C.c_int64()
        self._ck(self.lib.mr_get_step_history(self.h, 0, None, C.byref(n), 0))
        out = np.zeros(max(1, n.value), np.int32)
        self._ck(self.lib.mr_get_step_history(self.h, len(out), _ptr(out), C.byref(n), int(reset)))
        return out[:min(n.value, len(out))]

    def autotune(self, steps=5):
        best = C.c_int32()
        self._ck(self.lib.mr_autotune(self.h, steps, C.byref(best)))
        return best.value

    # ------------------------------------------------- learned proposal --
    CNN_PARAMS = 4961
    # parameter packing of the proposal network: W1, b1, W2, b2, W3, b3, wl, bl
    CNN_SHAPES = [(16, 2, 3, 3), (16,), (16, 16, 3, 3), (16,), (16, 16, 3, 3), (16,), (16,), (1,)]

    def set_tuning(self, ctas_per_sm=0, stage_form=-1):
        """Launch configuration: CTAs per SM (0 = occupancy) and the 2D stage form
        (1 warp per block, 0 CTA per block, -1 by block count)."""
        self._ck(self.lib.mr_set_tuning(self.h, ctas_per_sm, stage_form))

    def set_warp_form(self, blocks_per_cta=4, staging=1):
        """2D FP32 warp-per-block stage: warps (blocks) per CTA and bulk-copy staging of the rows."""
        self._ck(self.lib.mr_set_warp_form(self.h, blocks_per_cta, staging))

    def set_refine_mode(self, mode):
        self._ck(self.lib.mr_set_refine_mode(self.h, {"all": 0, "learned": 1}.get(mode, mode)))

    def proposal_collect(self, on=True, capacity=0):
        self._ck(self.lib.mr_proposal_collect(self.h, int(bool(on)), capacity))

    def proposal_dataset(self):
        n, p = C.c_int64(), C.c_int64()
        self._ck(self.lib.mr_proposal_dataset(self.h, C.byref(n), C.byref(p)))
        return n.value, p.value

    def proposal_train(self, init=None, epochs=5, batch=256, lr=1e-3, w_pos=4.0, recall=0.999,
                       holdout=0.2):
        tau, loss = C.c_float(), C.c_float()
        ini = None if init is None else np.ascontiguousarray(init, np.float32)
        self._ck(self.lib.mr_proposal_train(self.h, _ptr(ini), epochs, batch, lr, w_pos, recall, holdout,
                                            C.byref(tau), C.byref(loss)))
        return tau.value, loss.value

    def proposal_set(self, params=None, tau=0.5):
        pr = None if params is None else np.ascontiguousarray(params, np.float32)
        self._ck(self.lib.mr_proposal_set(self.h, _ptr(pr), tau))

    def proposal_get(self):
        w = np.zeros(self.CNN_PARAMS, np.float32)
        tau = C.c_float()
        self._ck(self.lib.mr_proposal_get(self.h, _ptr(w), C.byref(tau)))
        return w, tau.value

    def proposal_stats(self, reset=True):
        out = np.zeros(5, np.int64)
        self._ck(self.lib.mr_proposal_stats(self.h, _ptr(out), int(reset)))
        return dict(considered=int(out[0]), network=int(out[1]), fallback=int(out[2]),
                    misses=int(out[3]), closure=int(out[4]))

    def cnn_eval(self, params, x, y, w_pos=4.0):
        x = np.ascontiguousarray(x, np.float32)
        y = np.ascontiguousarray(y, np.float32)
        params = np.ascontiguousarray(params, np.float32)
        n = len(y)
        prob = np.zeros(n, np.float32)
        grad = np.zeros(self.CNN_PARAMS, np.float32)
        loss = C.c_float()
        self._ck(self.lib.mr_cnn_eval(self.h, _ptr(params), _ptr(x), _ptr(y), n, w_pos, _ptr(prob),
                                      _ptr(grad), C.byref(loss)))
        return prob, grad, loss.value

    def enable_timing(self, on=True):
        self._ck(self.lib.mr_enable_timing(self.h, int(bool(on))))

    def reset_stats(self):
        self._ck(self.lib.mr_reset_stats(self.h))

    def stats(self):
        s = Stats()
        self._ck(self.lib.mr_get_stats(self.h, C.byref(s)))
        return dict(ms={PHASES[i]: s.ms[i] for i in range(6)},
                    calls={PHASES[i]: s.phase_calls[i] for i in range(6)},
                    stage_launches=s.stage_launches, stage_blocks=s.stage_blocks, steps=s.steps,
                    det_launches=s.det_launches, det_blocks=s.det_blocks)
