"""ctypes binding of the C ABI in include/ncs.h (argument marshalling only).

Every computation runs in libncs.so (host precompute in C++, products and GMRES in
CUDA kernels). Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libncs.so")

NCS_OK = 0
NCS_E_INPUT = -1
NCS_E_NOCONV = -2
NCS_E_NUMERIC = -3
NCS_E_CUDA = -4
NCS_E_TIMEOUT = -5
NCS_E_OOM = -6
NCS_E_STATE = -7
EXTERIOR, INTERIOR = 0, 1
FP64, FP32, MIXED, DF64 = 0, 1, 2, 3
PRECISION_DEFAULT = -1  # the context precision set by Context.set_precision
METHOD_AUTO, METHOD_DIRECT, METHOD_TREE = 0, 1, 2

EXPORTS = ["ncs_default_params", "ncs_create", "ncs_create_from_operator", "ncs_info", "ncs_timings",
           "ncs_get_operator", "ncs_get_onepatch", "ncs_set_patches", "ncs_set_method", "ncs_matvec",
           "ncs_matvec_dev", "ncs_field_dev", "ncs_solve", "ncs_eval", "ncs_last_error", "ncs_destroy",
           "ncs_tree_pairs", "ncs_tree_stats", "ncs_profile_matvec", "ncs_create_from_operators", "ncs_get_reps",
           "ncs_tc_gemm_f32", "ncs_batch_solve", "ncs_block_dots", "ncs_block_dots_noalloc",
           "ncs_launch_count", "ncs_get_rep", "ncs_set_precision", "ncs_patch_residual", "ncs_solve_stats", "ncs_tune", "ncs_set_tuning",
           "ncs_get_tuning", "ncs_fma_peak"]


class ncs_params(ctypes.Structure):
    _fields_ = [("npan", ctypes.c_int), ("nord", ctypes.c_int), ("ntheta_fine", ctypes.c_int),
                ("id_tol", ctypes.c_double), ("threads", ctypes.c_int), ("grid_tol", ctypes.c_double),
                ("method", ctypes.c_int), ("tree_min_patches", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
                ("verbose", ctypes.c_int), ("mixed_residual", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("residual_update", ctypes.c_int), ("id_ladder_max", ctypes.c_double),
                ("device_precompute", ctypes.c_int), ("cuda_graphs", ctypes.c_int),
                ("batch_ladder_by_n", ctypes.c_int), ("batch_grouped", ctypes.c_int),
                ("inner_grid_tol", ctypes.c_double)]


class ncs_tuning(ctypes.Structure):
    _fields_ = [("p2l_tile", ctypes.c_int), ("p2l_poly", ctypes.c_int), ("direct_poly", ctypes.c_int),
                ("item_patches", ctypes.c_int), ("l2p_weight", ctypes.c_double), ("p2l_rsq", ctypes.c_int),
                ("direct_rsq", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NcsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ncs error {code}: {msg}")
        self.code = code


_lib = None
D = ctypes.POINTER(ctypes.c_double)
VP = ctypes.c_void_p


def load(path: str = LIB_PATH):
    """Loads libncs.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not built: run paper_1906_04209_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.ncs_default_params.argtypes = [ctypes.POINTER(ncs_params)]
    lib.ncs_default_params.restype = None
    lib.ncs_create.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ncs_params),
                               ctypes.POINTER(VP)]
    lib.ncs_create_from_operator.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D, D, D,
                                             ctypes.POINTER(ncs_params), ctypes.POINTER(VP)]
    lib.ncs_create_from_operators.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, D,
                                              ctypes.POINTER(ctypes.c_int), D, D, D, D, ctypes.POINTER(ncs_params),
                                              ctypes.POINTER(VP)]
    lib.ncs_get_reps.argtypes = [VP, ctypes.POINTER(ctypes.c_int), D, ctypes.POINTER(ctypes.c_int)]
    lib.ncs_info.argtypes = [VP, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    lib.ncs_timings.argtypes = [VP, D, ctypes.c_int]
    lib.ncs_get_operator.argtypes = [VP, D, D, D, D, D, D, D]
    lib.ncs_get_onepatch.argtypes = [VP, D, D]
    lib.ncs_set_patches.argtypes = [VP, ctypes.c_int64, D]
    lib.ncs_set_method.argtypes = [VP, ctypes.c_int]
    lib.ncs_matvec.argtypes = [VP, D, D, ctypes.c_int]
    lib.ncs_matvec_dev.argtypes = [VP, VP, VP, ctypes.c_int, VP]
    lib.ncs_field_dev.argtypes = [VP, VP, VP, ctypes.c_int, VP]
    lib.ncs_solve.argtypes = [VP, ctypes.c_double, ctypes.c_int, D, D, D, ctypes.POINTER(ctypes.c_int), D]
    lib.ncs_eval.argtypes = [VP, ctypes.c_int64, D, D, D]
    lib.ncs_last_error.argtypes = [VP]
    lib.ncs_last_error.restype = ctypes.c_char_p
    I32 = ctypes.POINTER(ctypes.c_int)
    lib.ncs_tree_pairs.argtypes = [VP, ctypes.POINTER(ctypes.c_int64), I32, I32, I32, I32]
    lib.ncs_tree_stats.argtypes = [VP, ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
    lib.ncs_profile_matvec.argtypes = [VP, VP, VP, ctypes.c_int, VP, D, ctypes.c_int]
    lib.ncs_tc_gemm_f32.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_int, VP, VP, VP, VP]
    lib.ncs_batch_solve.argtypes = [ctypes.c_int, D, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(D), ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(ncs_params), ctypes.c_int, D, D, ctypes.POINTER(ctypes.c_int), D,
                                    ctypes.POINTER(ctypes.c_int), D]
    lib.ncs_block_dots.argtypes = [ctypes.c_int64, ctypes.c_int, VP, ctypes.c_int64, VP, VP, VP]
    lib.ncs_block_dots_noalloc.argtypes = [ctypes.c_int64, ctypes.c_int, VP, ctypes.c_int64, VP, VP, VP]
    lib.ncs_get_rep.argtypes = [VP, ctypes.c_int, D, D, D]
    lib.ncs_set_precision.argtypes = [VP, ctypes.c_int]
    lib.ncs_solve_stats.argtypes = [VP, D, ctypes.c_int]
    lib.ncs_tune.argtypes = [VP, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ncs_tuning), D, ctypes.c_int]
    lib.ncs_set_tuning.argtypes = [VP, ctypes.POINTER(ncs_tuning)]
    lib.ncs_get_tuning.argtypes = [VP, ctypes.POINTER(ncs_tuning)]
    lib.ncs_fma_peak.argtypes = [ctypes.c_int, D]
    lib.ncs_launch_count.argtypes = []
    lib.ncs_launch_count.restype = ctypes.c_int64
    lib.ncs_destroy.argtypes = [VP]
    lib.ncs_destroy.restype = None
    for name in EXPORTS:
        if name not in ("ncs_default_params", "ncs_last_error", "ncs_destroy", "ncs_launch_count"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def tc_gemm_f32(rows, cols, kdim, A_ptr, B_ptr, D_ptr, stream=0):
    """D = A B^T on the tensor cores (see ncs_tc_gemm_f32); device pointers."""
    rc = load().ncs_tc_gemm_f32(rows, cols, kdim, VP(A_ptr), VP(B_ptr), VP(D_ptr), VP(stream))
    if rc != NCS_OK:
        raise NcsError(rc, "ncs_tc_gemm_f32 failed")


def batch_solve(instances, K, tol=1e-8, precision=MIXED, workers=0, **kw):
    """instances: list of (centres (N x 3), eps, mode). Returns a dict of per-instance
    arrays and timings (see ncs_batch_solve)."""
    lib = load()
    B = len(instances)
    eps = np.ascontiguousarray([e for _, e, _ in instances], dtype=np.float64)
    mode = np.ascontiguousarray([m for _, _, m in instances], dtype=np.int32)
    cs = [_f64(c).reshape(-1, 3) for c, _, _ in instances]
    N = np.ascontiguousarray([c.shape[0] for c in cs], dtype=np.int64)
    ptrs = (D * B)(*[c.ctypes.data_as(D) for c in cs])
    sc, Is, rr, secs = np.zeros(B), np.zeros(B), np.zeros(B), np.zeros(3)
    it, st = np.zeros(B, dtype=np.int32), np.zeros(B, dtype=np.int32)
    prm = default_params(**kw)
    I32 = ctypes.POINTER(ctypes.c_int)
    rc = lib.ncs_batch_solve(B, _ptr(eps), mode.ctypes.data_as(I32), N.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             ptrs, K, tol, precision, ctypes.byref(prm), workers, _ptr(sc), _ptr(Is),
                             it.ctypes.data_as(I32), _ptr(rr), st.ctypes.data_as(I32), _ptr(secs))
    return dict(rc=rc, scalar=sc, Isigma=Is, iterations=it, relres=rr, status=st, seconds=secs)


def block_dots(n, k, V_ptr, ld, w_ptr, out_ptr, stream=0):
    """out[j] = V_j . w on the device (see ncs_block_dots)."""
    rc = load().ncs_block_dots(n, k, VP(V_ptr), ld, VP(w_ptr), VP(out_ptr), VP(stream))
    if rc != NCS_OK:
        raise NcsError(rc, "ncs_block_dots failed")


def fma_peak(precision=FP64):
    """Measured FMA peak of the current device in TFLOP/s (see ncs_fma_peak)."""
    out = ctypes.c_double()
    rc = load().ncs_fma_peak(precision, ctypes.byref(out))
    if rc != NCS_OK:
        raise NcsError(rc, "ncs_fma_peak failed")
    return out.value


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(load().ncs_launch_count())


def block_dots_noalloc(n, k, V_ptr, ld, w_ptr, out_ptr, stream=0):
    """ncs_block_dots without allocating (fixed scratch, k <= 1024); asynchronous."""
    rc = load().ncs_block_dots_noalloc(n, k, VP(V_ptr), ld, VP(w_ptr), VP(out_ptr), VP(stream))
    if rc != NCS_OK:
        raise NcsError(rc, "ncs_block_dots_noalloc failed")


def default_params(**kw) -> ncs_params:
    p = ncs_params()
    load().ncs_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Context:
    """One solver context (precompute for (eps, mode, K) plus a patch layout)."""

    def __init__(self, eps, mode, K, params=None, operator=None, **kw):
        lib = load()
        prm = params or default_params(**kw)
        h = VP()
        if operator is None:
            rc = lib.ncs_create(eps, mode, K, ctypes.byref(prm), ctypes.byref(h))
        elif isinstance(operator, dict):
            # several representations: dict(rho_min=[...], reps=[(T, st, sth), ...], I=I)
            rm = _f64(operator["rho_min"])
            ps = np.ascontiguousarray([r[0].shape[0] for r in operator["reps"]], dtype=np.int32)
            T = _f64(np.concatenate([r[0] for r in operator["reps"]], axis=0))
            st = _f64(np.concatenate([r[1] for r in operator["reps"]]))
            sth = _f64(np.concatenate([r[2] for r in operator["reps"]]))
            I = _f64(operator["I"])
            rc = lib.ncs_create_from_operators(eps, mode, K, len(ps), _ptr(rm),
                                               ps.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _ptr(T), _ptr(st),
                                               _ptr(sth), _ptr(I), ctypes.byref(prm), ctypes.byref(h))
        else:
            T, st, sth, I = (_f64(a) for a in operator)
            p = T.shape[0]
            rc = lib.ncs_create_from_operator(eps, mode, K, p, _ptr(T), _ptr(st), _ptr(sth), _ptr(I),
                                              ctypes.byref(prm), ctypes.byref(h))
        if rc != NCS_OK:
            raise NcsError(rc, "ncs_create failed")
        self.h = h
        self.eps, self.mode, self.K = eps, mode, K
        self.N = 0

    def _check(self, rc):
        if rc != NCS_OK:
            raise NcsError(rc, load().ncs_last_error(self.h).decode())
        return rc

    def close(self):
        if self.h:
            load().ncs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        out = (ctypes.c_int64 * 13)()
        load().ncs_info(self.h, out, 13)
        keys = ["K", "Kstar", "p", "M", "nf", "N", "nrad", "levels", "grid_points", "tree_pairs", "direct_pairs",
                "inner_grid_points", "inner_tree_pairs"]
        return dict(zip(keys, [int(v) for v in out]))

    def timings(self):
        """[one-patch s, ID s, 1 if the ID ran on the device, sketch s, CPQR s,
        T assembly s, 1 if the collocation matrices were formed on the device,
        collocation s, LU + modal solves s]"""
        out = np.zeros(9)
        load().ncs_timings(self.h, _ptr(out), 9)
        return out

    def operator(self):
        i = self.info()
        T = np.zeros((i["p"], i["K"]))
        st, sth = np.zeros(i["p"]), np.zeros(i["p"])
        I = np.zeros(i["K"])
        P = np.zeros((i["K"], i["Kstar"]))
        zr, zth = np.zeros(i["Kstar"]), np.zeros(i["Kstar"])
        self._check(load().ncs_get_operator(self.h, _ptr(T), _ptr(st), _ptr(sth), _ptr(I), _ptr(P), _ptr(zr),
                                            _ptr(zth)))
        return dict(T=T, skel_t=st, skel_theta=sth, I=I, P=P, znode_r=zr, znode_theta=zth)

    def reps(self):
        """(far-field radii, ranks) of the outgoing representations."""
        lib = load()
        n = ctypes.c_int(0)
        self._check(lib.ncs_get_reps(self.h, ctypes.byref(n), None, None))
        rm = np.zeros(n.value)
        ps = np.zeros(n.value, dtype=np.int32)
        self._check(lib.ncs_get_reps(self.h, ctypes.byref(n), _ptr(rm), ps.ctypes.data_as(ctypes.POINTER(ctypes.c_int))))
        return rm, ps

    def set_precision(self, precision):
        """Context precision used by calls given PRECISION_DEFAULT."""
        self._check(load().ncs_set_precision(self.h, precision))

    def rep(self, r):
        """(T, skel_t, skel_theta) of outgoing representation r."""
        rm, ps = self.reps()
        p = int(ps[r])
        T, st, sth = np.zeros((p, self.K)), np.zeros(p), np.zeros(p)
        self._check(load().ncs_get_rep(self.h, r, _ptr(T), _ptr(st), _ptr(sth)))
        return T, st, sth

    def onepatch(self):
        i = self.info()
        tr = np.zeros(i["nrad"])
        beta = np.zeros((i["nrad"], i["K"]))
        self._check(load().ncs_get_onepatch(self.h, _ptr(tr), _ptr(beta)))
        return tr, beta

    def set_patches(self, centres):
        c = _f64(centres).reshape(-1, 3)
        self._check(load().ncs_set_patches(self.h, c.shape[0], _ptr(c)))
        self.N = c.shape[0]

    def tree_pairs(self):
        """(target, source, level, kind) arrays of every pair the tree accounts for."""
        lib = load()
        n = ctypes.c_int64(0)
        self._check(lib.ncs_tree_pairs(self.h, ctypes.byref(n), None, None, None, None))
        arrs = [np.zeros(n.value, dtype=np.int32) for _ in range(4)]
        ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) for a in arrs]
        self._check(lib.ncs_tree_pairs(self.h, ctypes.byref(n), *ptrs))
        return tuple(arrs)

    def tree_stats(self) -> dict:
        out = (ctypes.c_int64 * 11)()
        self._check(load().ncs_tree_stats(self.h, out, 11))
        keys = ["levels", "grid_groups", "grid_points", "p2l_items", "p2l_pairs", "direct_pairs", "l2p_evals",
                "direct_patch_pairs", "shapes", "l2l_links", "l2l_evals"]
        return dict(zip(keys, [int(v) for v in out]))

    def set_method(self, method):
        self._check(load().ncs_set_method(self.h, method))

    def matvec(self, x, precision=FP64):
        x = _f64(x).ravel()
        y = np.empty_like(x)
        self._check(load().ncs_matvec(self.h, _ptr(x), _ptr(y), precision))
        return y

    def matvec_dev(self, x_ptr, y_ptr, precision=FP64, stream=0):
        """x_ptr, y_ptr: device addresses (e.g. torch tensor.data_ptr())."""
        self._check(load().ncs_matvec_dev(self.h, VP(x_ptr), VP(y_ptr), precision, VP(stream)))

    def profile_matvec(self, x_ptr, y_ptr, precision=FP64, stream=0):
        """Per-stage milliseconds of one product (see ncs_profile_matvec)."""
        ms = np.zeros(7)
        self._check(load().ncs_profile_matvec(self.h, VP(x_ptr), VP(y_ptr), precision, VP(stream), _ptr(ms), 7))
        return dict(zip(["outgoing", "p2l", "coef", "direct", "l2p", "apply_P", "total"], ms.tolist()))

    def field_dev(self, x_ptr, z_ptr, precision=FP64, stream=0):
        self._check(load().ncs_field_dev(self.h, VP(x_ptr), VP(z_ptr), precision, VP(stream)))

    def solve(self, tol=1e-10, precision=FP64, want_fhat=True, allow_noconv=False):
        fhat = np.zeros(self.N * self.K) if want_fhat else None
        sc, Is, rr = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        it = ctypes.c_int()
        rc = load().ncs_solve(self.h, tol, precision, _ptr(fhat), ctypes.byref(sc), ctypes.byref(Is),
                              ctypes.byref(it), ctypes.byref(rr))
        if rc != NCS_OK and not (allow_noconv and rc == NCS_E_NOCONV):
            self._check(rc)
        return dict(fhat=fhat, scalar=sc.value, Isigma=Is.value, iterations=it.value, relres=rr.value, rc=rc)

    def tune(self, flags=3, cache_path=None):
        """Picks the tree product's launch configuration for this layout (see ncs_tune).
        Returns (configuration dict, report dict)."""
        t = ncs_tuning()
        rep = np.zeros(6)
        cp = None if cache_path is None else os.fsencode(cache_path)
        self._check(load().ncs_tune(self.h, flags, cp, ctypes.byref(t), _ptr(rep), 6))
        keys = ["default_ms", "tuned_ms", "trial_products", "error", "seconds", "from_cache"]
        return t.as_dict(), dict(zip(keys, rep.tolist()))

    def set_tuning(self, **kw):
        t = ncs_tuning()
        self._check(load().ncs_get_tuning(self.h, ctypes.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        self._check(load().ncs_set_tuning(self.h, ctypes.byref(t)))

    def get_tuning(self) -> dict:
        t = ncs_tuning()
        self._check(load().ncs_get_tuning(self.h, ctypes.byref(t)))
        return t.as_dict()

    def solve_stats(self) -> dict:
        """Counters of the last solve (see ncs_solve_stats)."""
        out = np.zeros(8)
        self._check(load().ncs_solve_stats(self.h, _ptr(out), 8))
        keys = ["gmres_steps", "residual_products", "residual_updates", "refinement_steps", "relres",
                "graph_replays", "seconds", "recomputed"]
        return dict(zip(keys, out.tolist()))

    def eval(self, targets, fhat):
        t = _f64(targets).reshape(-1, 3)
        f = _f64(fhat).ravel()
        out = np.zeros(t.shape[0])
        self._check(load().ncs_eval(self.h, t.shape[0], _ptr(t), _ptr(f), _ptr(out)))
        return out

    def patch_residual(self, i, fhat, nt=0, nth=0):
        """Relative L2 residual of the system on patch i (eq. l2res)."""
        f = _f64(fhat).ravel()
        out = ctypes.c_double()
        self._check(load().ncs_patch_residual(self.h, ctypes.c_int64(i), _ptr(f), nt, nth, ctypes.byref(out)))
        return out.value
