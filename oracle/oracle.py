"""ctypes wrapper around the FP64 C oracle (``fewha_oracle.c``).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The geometry argument is any object with the attributes ``D``, ``obstruction``,
``n_sub``, ``gs`` (sequence of objects with ``theta_x``, ``theta_y``, ``H``),
``layers`` (objects with ``h``, ``cn2``, ``n``, ``J``, ``delta``), ``r0``,
``alpha`` and ``wavelet_N``.  Noise weights (1/sigma_g^2) are passed
separately.  Arrays in and out are float64 numpy arrays.
"""
import ctypes as C
import os
import subprocess
import threading

import numpy as np

from .daubechies import daubechies_taps

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fewha_oracle.c")
_LIB = os.path.join(_HERE, "libfewha_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def oracle_lib_path() -> str:
    return _LIB


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [("D", C.c_double), ("obstruction", C.c_double), ("n_sub", C.c_int),
                ("n_gs", C.c_int), ("gs_tx", _dp), ("gs_ty", _dp), ("gs_H", _dp), ("gs_w", _dp),
                ("n_layers", C.c_int), ("lay_h", _dp), ("lay_cn2", _dp), ("lay_delta", _dp),
                ("lay_n", _ip), ("lay_J", _ip), ("r0", C.c_double), ("alpha", C.c_double),
                ("n_taps", C.c_int), ("taps", _dp), ("gs_ns", _ip)]


class _Opts(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("rtol", C.c_double), ("augmented", C.c_int),
                ("init_mode", C.c_int), ("loop_mode", C.c_int), ("true_residual_init", C.c_int),
                ("true_res_every", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_res", C.c_double), ("bnorm", C.c_double),
                ("status", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle()
            lib = C.CDLL(_LIB)
            vp = C.c_void_p
            lib.orc_create.argtypes = [C.POINTER(_Params), C.c_int, C.POINTER(vp)]
            lib.orc_create.restype = C.c_int
            lib.orc_destroy.argtypes = [vp]
            lib.orc_n_unknowns.argtypes = [vp]
            lib.orc_n_unknowns.restype = C.c_long
            lib.orc_n_slopes.argtypes = [vp]
            lib.orc_n_slopes.restype = C.c_long
            lib.orc_layer_spacing.argtypes = [vp, C.c_int]
            lib.orc_layer_spacing.restype = C.c_double
            lib.orc_mask.argtypes = [vp]
            lib.orc_mask.restype = C.POINTER(C.c_ubyte)
            lib.orc_prior.argtypes = [vp]
            lib.orc_prior.restype = _dp
            lib.orc_invJ.argtypes = [vp]
            lib.orc_invJ.restype = _dp
            lib.orc_set_invJ.argtypes = [vp, _dp]
            for name in ("orc_apply_op", "orc_rhs", "orc_apply_A", "orc_apply_AT"):
                getattr(lib, name).argtypes = [vp, _dp, _dp]
            lib.orc_apply_Cinv.argtypes = [vp, _dp]
            lib.orc_prop_fwd.argtypes = [vp, C.c_int, _dp, _dp]
            lib.orc_prop_adj.argtypes = [vp, C.c_int, _dp, _dp]
            lib.orc_gamma_fwd.argtypes = [C.c_int, _dp, _dp]
            lib.orc_gamma_adj.argtypes = [C.c_int, _dp, _dp]
            lib.orc_dwt1_fwd.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
            lib.orc_dwt1_inv.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp]
            lib.orc_dwt2_fwd.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
            lib.orc_dwt2_inv.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
            lib.orc_band_of.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _ip, _ip]
            lib.orc_data_diag.argtypes = [vp, C.c_long]
            lib.orc_data_diag.restype = C.c_double
            lib.orc_dense_M.argtypes = [vp, _dp]
            lib.orc_solve.argtypes = [vp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, C.c_int, _ip,
                                      C.POINTER(_Opts), C.POINTER(_Stats), _dp]
            lib.orc_solve.restype = C.c_int
            lib.orc_fit.argtypes = [vp, _dp, _dp]
            lib.orc_fit.restype = C.c_int
            lib.orc_pol_slopes.argtypes = [vp, _dp, _dp, _dp]
            lib.orc_pol_slopes.restype = C.c_int
            lib.orc_slope_offset.argtypes = [vp, C.c_int]
            lib.orc_slope_offset.restype = C.c_long
            lib.orc_sensor_ns.argtypes = [vp, C.c_int]
            lib.orc_sensor_ns.restype = C.c_int
            lib.orc_control.argtypes = [C.c_long, C.c_int, C.c_double, _dp, _dp, _dp, _dp]
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# Stand-alone 1-D / 2-D wavelet transforms (Sec. 3)
# ---------------------------------------------------------------------------

def dwt1_fwd(x, taps):
    lib = _load()
    x, taps = _f64(x), _f64(taps)
    out = np.empty_like(x)
    lib.orc_dwt1_fwd(len(x), len(taps), _ptr(taps), _ptr(x), _ptr(out))
    return out


def dwt1_inv(ad, taps):
    lib = _load()
    ad, taps = _f64(ad), _f64(taps)
    out = np.empty_like(ad)
    lib.orc_dwt1_inv(len(ad), len(taps), _ptr(taps), _ptr(ad), _ptr(out))
    return out


def dwt2_fwd(x, J, taps):
    lib = _load()
    x, taps = _f64(x), _f64(taps)
    out = np.empty_like(x)
    lib.orc_dwt2_fwd(x.shape[0], J, len(taps), _ptr(taps), _ptr(x), _ptr(out))
    return out


def dwt2_inv(c, J, taps):
    lib = _load()
    c, taps = _f64(c), _f64(taps)
    out = np.empty_like(c)
    lib.orc_dwt2_inv(c.shape[0], J, len(taps), _ptr(taps), _ptr(c), _ptr(out))
    return out


def gamma_fwd(wf):
    lib = _load()
    wf = _f64(wf)
    ns = wf.shape[0] - 1
    s = np.empty(2 * ns * ns)
    lib.orc_gamma_fwd(ns, _ptr(wf), _ptr(s))
    return s


def gamma_adj(s, ns):
    lib = _load()
    s = _f64(s)
    wf = np.zeros((ns + 1, ns + 1))
    lib.orc_gamma_adj(ns, _ptr(s), _ptr(wf))
    return wf


def band_of(n, J, r, q):
    lib = _load()
    s, quad = C.c_int(), C.c_int()
    lib.orc_band_of(n, J, r, q, C.byref(s), C.byref(quad))
    return s.value, quad.value


class Oracle:
    """FP64 oracle context for one geometry (Sec. 2-4)."""

    INIT_GRAM, INIT_PAPER = 0, 1
    LOOP_LAST, LOOP_ALL = 0, 1

    def __init__(self, geom, noise_w, with_precond=True, taps=None):
        lib = _load()
        self._lib = lib
        gs, lays = list(geom.gs), list(geom.layers)
        self._keep = []

        def arr(vals, dt=np.float64):
            a = np.ascontiguousarray(np.asarray(vals, dtype=dt))
            self._keep.append(a)
            return a

        self.taps = arr(daubechies_taps(geom.wavelet_N) if taps is None else taps)
        tx, ty = arr([g.theta_x for g in gs]), arr([g.theta_y for g in gs])
        H, w = arr([g.H for g in gs]), arr(noise_w)
        lh, lc = arr([l.h for l in lays]), arr([l.cn2 for l in lays])
        ld = arr([l.delta for l in lays])
        ln = arr([l.n for l in lays], np.int32)
        lJ = arr([l.J for l in lays], np.int32)
        gns = arr([getattr(g, "n_sub", 0) or geom.n_sub for g in gs], np.int32)
        ip = lambda a: a.ctypes.data_as(_ip)  # noqa: E731
        self._p = _Params(geom.D, geom.obstruction, geom.n_sub, len(gs), _ptr(tx), _ptr(ty),
                          _ptr(H), _ptr(w), len(lays), _ptr(lh), _ptr(lc), _ptr(ld), ip(ln), ip(lJ),
                          geom.r0, geom.alpha, len(self.taps), _ptr(self.taps), ip(gns))
        h = C.c_void_p()
        st = lib.orc_create(C.byref(self._p), 1 if with_precond else 0, C.byref(h))
        if st != 0:
            raise ValueError("oracle geometry rejected (status %d)" % st)
        self._h = h
        self.geom = geom
        self.n = lib.orc_n_unknowns(h)
        self.n_slopes = lib.orc_n_slopes(h)
        self.n_sub = geom.n_sub
        self.sensor_ns = [lib.orc_sensor_ns(h, g) for g in range(len(gs))]
        self.slope_off = [lib.orc_slope_offset(h, g) for g in range(len(gs))] + [self.n_slopes]
        self.layer_n = [l.n for l in lays]
        self.layer_off = np.concatenate([[0], np.cumsum([l.n * l.n for l in lays])]).astype(int)

    def __del__(self):
        if getattr(self, "_h", None) is not None:
            self._lib.orc_destroy(self._h)
            self._h = None

    # -- geometry / tables --------------------------------------------------
    def layer_spacing(self, l):
        return self._lib.orc_layer_spacing(self._h, l)

    def mask(self, g=0):
        """Lit subapertures of guide star g's sensor (n_g^2 booleans)."""
        off = sum(n * n for n in self.sensor_ns[:g])
        m = np.ctypeslib.as_array(self._lib.orc_mask(self._h), shape=(off + self.sensor_ns[g] ** 2,))
        return m[off:].copy().astype(bool)

    def prior(self):
        return np.ctypeslib.as_array(self._lib.orc_prior(self._h), shape=(self.n,)).copy()

    def invJ(self):
        return np.ctypeslib.as_array(self._lib.orc_invJ(self._h), shape=(self.n,)).copy()

    def set_invJ(self, invJ):
        invJ = _f64(invJ)
        self._lib.orc_set_invJ(self._h, _ptr(invJ))

    def data_diag(self, i):
        return self._lib.orc_data_diag(self._h, int(i))

    # -- operators ----------------------------------------------------------
    def _unary(self, name, x, nout):
        x = _f64(x)
        y = np.empty(nout)
        getattr(self._lib, name)(self._h, _ptr(x), _ptr(y))
        return y

    def apply_op(self, x):
        return self._unary("orc_apply_op", x, self.n)

    # -- mirror side of Algorithm 3 (one ground DM on the pupil nodes) -------
    @property
    def n_actuators(self):
        return (self.n_sub + 1) ** 2

    def fit(self, c):
        """a~ = F W^{-1} c (on-axis projection of the layers onto the actuators)."""
        c = _f64(c)
        a = np.zeros(self.n_actuators)
        st = self._lib.orc_fit(self._h, _ptr(c), _ptr(a))
        if st != 0:
            raise ValueError("fitting direction outside a layer grid")
        return a

    def pol_slopes(self, s, a):
        """s + Gamma a for every guide star (pseudo-open-loop measurements)."""
        s, a = _f64(s), _f64(a)
        out = np.zeros_like(s)
        if self._lib.orc_pol_slopes(self._h, _ptr(s), _ptr(a), _ptr(out)) != 0:
            raise ValueError("pseudo-open-loop slopes need every sensor on the mirror's grid")
        return out

    def control(self, closed, gain, a_im1, a_i, a_fit):
        """Gain control of Algorithm 3 (closed or open loop)."""
        a_im1, a_i, a_fit = _f64(a_im1), _f64(a_i), _f64(a_fit)
        out = np.zeros_like(a_i)
        self._lib.orc_control(a_i.size, 1 if closed else 0, float(gain), _ptr(a_im1), _ptr(a_i),
                              _ptr(a_fit), _ptr(out))
        return out

    def rhs(self, s):
        return self._unary("orc_rhs", s, self.n)

    def apply_A(self, nodal):
        return self._unary("orc_apply_A", nodal, self.n_slopes)

    def apply_AT(self, s):
        return self._unary("orc_apply_AT", s, self.n)

    def apply_Cinv(self, s):
        s = _f64(s).copy()
        self._lib.orc_apply_Cinv(self._h, _ptr(s))
        return s

    def prop_fwd(self, g, nodal):
        nodal = _f64(nodal)
        wf = np.empty((self.sensor_ns[g] + 1) ** 2)
        self._lib.orc_prop_fwd(self._h, g, _ptr(nodal), _ptr(wf))
        return wf

    def prop_adj(self, g, wf):
        wf = _f64(wf)
        nodal = np.zeros(self.n)
        self._lib.orc_prop_adj(self._h, g, _ptr(wf), _ptr(nodal))
        return nodal

    def dense_M(self):
        M = np.empty((self.n, self.n))
        self._lib.orc_dense_M(self._h, _ptr(M))
        return M

    # -- one reconstructor time step (Algorithm 3 RHS/residual + Alg. 1/2) --
    def new_state(self, kcap):
        n = self.n
        return {"c": np.zeros(n), "b_prev": np.zeros(n), "r_prev": np.zeros(n),
                "P": np.zeros((kcap, n)), "Q": np.zeros((kcap, n)), "pq": np.zeros(kcap),
                "k_valid": 0, "kcap": kcap}

    def solve(self, s, state, max_iter, rtol=0.0, augmented=True, init_mode=0, loop_mode=0,
              true_residual_init=False, history=False, true_res_every=0):
        """Advance ``state`` (dict from ``new_state``) by one time step in place.
        ``true_res_every`` = N > 0 replaces the recurrence residual by b - M c
        after every N-th iteration."""
        s = _f64(s)
        for k in ("c", "b_prev", "r_prev", "P", "Q", "pq"):
            state[k] = _f64(state[k])
        kv = C.c_int(state["k_valid"])
        o = _Opts(max_iter, rtol, 1 if augmented else 0, init_mode, loop_mode,
                  1 if true_residual_init else 0, int(true_res_every))
        stt = _Stats()
        hist = np.zeros((4, max_iter + 1, self.n)) if history else None
        st = self._lib.orc_solve(self._h, _ptr(s), _ptr(state["c"]), _ptr(state["b_prev"]),
                                 _ptr(state["r_prev"]), _ptr(state["P"]), _ptr(state["Q"]),
                                 _ptr(state["pq"]), state["kcap"], C.byref(kv), C.byref(o),
                                 C.byref(stt), _ptr(hist) if history else None)
        state["k_valid"] = kv.value
        out = {"status": st, "iterations": stt.iterations, "rel_res": stt.rel_res,
               "bnorm": stt.bnorm}
        if history:
            out["history"] = {"r": hist[0], "z": hist[1], "p": hist[2], "q": hist[3]}
        return out
