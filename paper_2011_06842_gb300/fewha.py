"""Python binding of libfewha (include/fewha.h): argument marshalling only.

Every computation runs in the CUDA library; this module builds the C
structures, passes device pointers of torch tensors and the current CUDA
stream, and turns status codes into exceptions.  There is no fallback: if
libfewha.so is missing or no GPU is present the calls raise.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfewha.so")

MAX_GS, MAX_LAYERS, MAX_K, MAX_ITER = 16, 16, 16, 1000
F64, F32, BF16S = 0, 1, 2
RECYCLE_LAST, RECYCLE_ALL = 0, 1
LAUNCH_PERSISTENT, LAUNCH_PHASES = 0, 1
PRECISIONS = {"f64": F64, "f32": F32, "bf16s": BF16S}

ERRORS = {0: "ok", -1: "FEWHA_ERR_ARG", -2: "FEWHA_ERR_GEOMETRY", -3: "FEWHA_ERR_CUDA",
          -4: "FEWHA_ERR_TIMEOUT", -5: "FEWHA_ERR_BREAKDOWN", -6: "FEWHA_ERR_NOT_SPD",
          -7: "FEWHA_ERR_NOMEM", -8: "FEWHA_ERR_SCRATCH"}


class FewhaError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, ERRORS.get(status, "?"), status))


class GS(C.Structure):
    _fields_ = [("theta_x", C.c_double), ("theta_y", C.c_double), ("H", C.c_double),
                ("weight", C.c_double), ("n_sub", C.c_int), ("pad", C.c_int)]


class LAYER(C.Structure):
    _fields_ = [("h", C.c_double), ("cn2", C.c_double), ("delta", C.c_double), ("n", C.c_int),
                ("J", C.c_int)]


class GEOMETRY(C.Structure):
    _fields_ = [("D", C.c_double), ("obstruction", C.c_double), ("n_sub", C.c_int),
                ("n_gs", C.c_int), ("gs", GS * MAX_GS), ("n_layers", C.c_int),
                ("layers", LAYER * MAX_LAYERS), ("r0", C.c_double), ("alpha", C.c_double),
                ("wavelet_N", C.c_int), ("precision", C.c_int), ("tile", C.c_int), ("grid", C.c_int)]


class STATE(C.Structure):
    _fields_ = [("b_prev", C.c_void_p), ("r_prev", C.c_void_p), ("basis_P", C.c_void_p),
                ("basis_Q", C.c_void_p), ("basis_pq", C.c_void_p), ("meta", C.c_void_p),
                ("k_cap", C.c_int)]


class OPTS(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("rtol", C.c_double), ("augmented", C.c_int),
                ("recycle_mode", C.c_int), ("launch_mode", C.c_int), ("true_res_every", C.c_int),
                ("rhs_in_state", C.c_int), ("pad", C.c_int), ("c_out", C.c_void_p)]


class LAUNCH_INFO(C.Structure):
    _fields_ = [("ctas", C.c_int), ("threads", C.c_int), ("smem_bytes", C.c_long),
                ("split_levels", C.c_int), ("staged_tables", C.c_int), ("wfs_tile_y", C.c_int),
                ("wfs_tile_x", C.c_int), ("pt_bands", C.c_int), ("pt_rows_chunk", C.c_int),
                ("pt_rows_large", C.c_int), ("pt_rows_small", C.c_int)]


class STATS(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("rel_res", C.c_double),
                ("bnorm", C.c_double), ("rz", C.c_double), ("basis_count", C.c_int),
                ("pad", C.c_int)]


STATS_BYTES = C.sizeof(STATS)
_lib = None


def load_library(path=LIB_PATH):
    """Loads libfewha.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libfewha.so not found at %s: run paper_2011_06842_gb300.build.build()" % path)
    lib = C.CDLL(path)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    lib.fewha_create.argtypes = [C.POINTER(GEOMETRY), C.POINTER(vp)]
    lib.fewha_create.restype = C.c_int
    lib.fewha_destroy.argtypes = [vp]
    lib.fewha_destroy.restype = None
    lib.fewha_n_unknowns.argtypes = [vp]
    lib.fewha_n_unknowns.restype = C.c_long
    lib.fewha_n_slopes.argtypes = [vp]
    lib.fewha_n_slopes.restype = C.c_long
    lib.fewha_layer_spacing.argtypes = [vp, C.c_int]
    lib.fewha_layer_spacing.restype = C.c_double
    lib.fewha_read_probe.argtypes = [vp, C.c_long, C.c_int, vp, vp]
    lib.fewha_read_probe.restype = C.c_int
    lib.fewha_store.argtypes = [vp, vp, C.c_long, vp]
    lib.fewha_store.restype = C.c_int
    lib.fewha_set_pt_bands.argtypes = [vp, C.c_int, C.c_int]
    lib.fewha_set_pt_bands.restype = C.c_int
    lib.fewha_set_noise.argtypes = [vp, dp, C.c_int]
    lib.fewha_set_noise.restype = C.c_int
    lib.fewha_get_launch_info.argtypes = [vp, C.POINTER(LAUNCH_INFO)]
    lib.fewha_get_launch_info.restype = C.c_int
    lib.fewha_get_prior.argtypes = [vp, dp]
    lib.fewha_get_precond.argtypes = [vp, dp]
    lib.fewha_apply_op.argtypes = [vp, vp, vp, vp]
    lib.fewha_rhs.argtypes = [vp, vp, vp, vp]
    lib.fewha_solve.argtypes = [vp, vp, vp, C.POINTER(STATE), C.POINTER(OPTS), vp, vp]
    lib.fewha_apply_op_noalloc.argtypes = [vp, vp, vp, vp]
    lib.fewha_apply_op_noalloc.restype = C.c_int
    lib.fewha_set_timeout.argtypes = [vp, C.c_ulonglong]
    lib.fewha_set_timeout.restype = C.c_int
    lib.fewha_set_trace.argtypes = [vp, vp, C.c_int]
    lib.fewha_set_trace.restype = C.c_int
    lib.fewha_batch_create.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(C.c_int), C.POINTER(vp)]
    lib.fewha_batch_create.restype = C.c_int
    lib.fewha_batch_create_rounds.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                              C.POINTER(vp)]
    lib.fewha_batch_create_rounds.restype = C.c_int
    lib.fewha_batch_ctas.argtypes = [vp, C.POINTER(C.c_int)]
    lib.fewha_batch_ctas.restype = C.c_int
    lib.fewha_batch_tiles.argtypes = [vp, C.POINTER(C.c_int)]
    lib.fewha_batch_tiles.restype = C.c_int
    lib.fewha_batch_create_ex.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                          C.POINTER(C.c_int), C.POINTER(vp)]
    lib.fewha_batch_create_ex.restype = C.c_int
    lib.fewha_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(STATE), C.POINTER(OPTS), vp, vp]
    lib.fewha_batch_solve.restype = C.c_int
    lib.fewha_batch_bind.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(STATE), C.POINTER(OPTS), vp]
    lib.fewha_batch_bind.restype = C.c_int
    lib.fewha_batch_launch.argtypes = [vp, vp]
    lib.fewha_batch_launch.restype = C.c_int
    lib.fewha_batch_destroy.argtypes = [vp]
    lib.fewha_batch_destroy.restype = None
    lib.fewha_mcao_create.argtypes = [vp, vp, C.POINTER(vp)]
    lib.fewha_mcao_create.restype = C.c_int
    lib.fewha_mcao_n_actuators.argtypes = [vp]
    lib.fewha_mcao_n_actuators.restype = C.c_long
    lib.fewha_mcao_fit.argtypes = [vp, vp, vp, C.c_int, vp]
    lib.fewha_mcao_fit.restype = C.c_int
    lib.fewha_mcao_destroy.argtypes = [vp]
    lib.fewha_mcao_destroy.restype = None
    lib.fewha_n_actuators.argtypes = [vp]
    lib.fewha_n_actuators.restype = C.c_long
    lib.fewha_fit.argtypes = [vp, vp, vp, vp]
    lib.fewha_fit.restype = C.c_int
    lib.fewha_pol_slopes.argtypes = [vp, vp, vp, vp, vp]
    lib.fewha_pol_slopes.restype = C.c_int
    lib.fewha_control.argtypes = [vp, C.c_int, C.c_double, vp, vp, vp, vp, vp]
    lib.fewha_control.restype = C.c_int
    lib.fewha_apply_op_multi.argtypes = [vp, vp, C.c_long, vp, C.c_long, C.c_int, vp]
    lib.fewha_apply_op_multi.restype = C.c_int
    # learned warm start (float pointers as void*, strides and sizes as long/int)
    L, I, F = C.c_long, C.c_int, C.c_float
    learned = {
        "fewha_conv3x3_fwd": [vp, L, L, I, vp, vp, vp, L, L, I, I, I, I, I, vp],
        "fewha_conv3x3_fwd_tc": [vp, L, L, I, vp, vp, vp, L, L, I, I, I, I, I, vp, vp],
        "fewha_conv3x3_bwd_data": [vp, L, L, I, vp, vp, L, L, I, I, I, I, vp],
        "fewha_conv3x3_bwd_weight": [vp, L, L, I, vp, L, L, I, I, I, I, vp, vp, I, vp, vp],
        "fewha_relu_bwd": [vp, vp, L, vp],
        "fewha_mse_grad": [vp, vp, vp, L, vp, vp],
        "fewha_adam_step": [vp, vp, vp, vp, L, F, F, F, F, I, vp],
        "fewha_scale": [vp, vp, vp, L, I, vp],
        "fewha_learned_targets": [vp, vp, vp, vp, vp, L, vp],
        "fewha_deflate_warm_start": [vp, vp, L, vp, L, I, vp, vp, vp, L, vp, vp, vp, vp],
    }
    for name, args in learned.items():
        getattr(lib, name).argtypes = args
        getattr(lib, name).restype = C.c_int
    lib.fewha_conv3x3_wgrad_workspace.argtypes = [I, I, I, I, I]
    lib.fewha_conv3x3_wgrad_workspace.restype = C.c_long
    lib.fewha_strerror.argtypes = [C.c_int]
    lib.fewha_strerror.restype = C.c_char_p
    for name in ("fewha_create", "fewha_get_prior", "fewha_get_precond", "fewha_apply_op",
                 "fewha_rhs", "fewha_solve"):
        getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def exported_symbols():
    """Entry points declared in include/fewha.h."""
    return ["fewha_create", "fewha_destroy", "fewha_n_unknowns", "fewha_n_slopes",
            "fewha_layer_spacing", "fewha_get_prior", "fewha_get_precond", "fewha_apply_op",
            "fewha_rhs", "fewha_solve", "fewha_set_timeout", "fewha_set_trace", "fewha_apply_op_noalloc", "fewha_batch_create",
            "fewha_batch_ctas", "fewha_batch_solve", "fewha_batch_destroy", "fewha_strerror",
            "fewha_batch_bind", "fewha_batch_launch", "fewha_batch_create_rounds", "fewha_n_actuators", "fewha_fit",
            "fewha_pol_slopes", "fewha_control",
            "fewha_apply_op_multi", "fewha_conv3x3_fwd", "fewha_conv3x3_bwd_data",
            "fewha_conv3x3_wgrad_workspace", "fewha_conv3x3_bwd_weight", "fewha_relu_bwd",
            "fewha_mse_grad", "fewha_adam_step", "fewha_scale", "fewha_learned_targets",
            "fewha_deflate_warm_start", "fewha_mcao_create", "fewha_mcao_n_actuators", "fewha_mcao_fit",
            "fewha_mcao_destroy", "fewha_get_launch_info", "fewha_set_noise", "fewha_read_probe", "fewha_set_pt_bands",
            "fewha_batch_create_ex", "fewha_batch_tiles", "fewha_conv3x3_fwd_tc", "fewha_store"]


def make_geometry(geom, noise_w, precision="f64", tile=0, grid=0) -> GEOMETRY:
    """C geometry from a description object (attributes D, obstruction, n_sub,
    gs[theta_x, theta_y, H], layers[h, cn2, n, J, delta], r0, alpha, wavelet_N)."""
    g = GEOMETRY()
    g.D, g.obstruction, g.n_sub = geom.D, geom.obstruction, geom.n_sub
    if len(geom.gs) > MAX_GS or len(geom.layers) > MAX_LAYERS:
        raise ValueError("too many guide stars or layers")
    g.n_gs = len(geom.gs)
    for i, (s, w) in enumerate(zip(geom.gs, noise_w)):
        g.gs[i] = GS(s.theta_x, s.theta_y, s.H, float(w), int(getattr(s, "n_sub", 0) or 0), 0)
    g.n_layers = len(geom.layers)
    for i, l in enumerate(geom.layers):
        g.layers[i] = LAYER(l.h, l.cn2, l.delta, l.n, l.J)
    g.r0, g.alpha, g.wavelet_N = geom.r0, geom.alpha, geom.wavelet_N
    g.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    g.tile, g.grid = tile, grid
    return g


def _stream_ptr(torch):
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class FewhaState:
    """Caller-owned per-time-step state (device tensors) of fewha_solve."""

    def __init__(self, torch, n, kcap, dtype, device):
        if not 1 <= kcap <= MAX_K:
            raise ValueError("k_cap must be in 1..%d" % MAX_K)
        self.kcap = kcap
        self.b_prev = torch.zeros(n, dtype=dtype, device=device)
        self.r_prev = torch.zeros(n, dtype=dtype, device=device)
        self.P = torch.zeros((2, kcap, n), dtype=dtype, device=device)
        self.Q = torch.zeros((2, kcap, n), dtype=dtype, device=device)
        self.pq = torch.zeros((2, kcap), dtype=torch.float64, device=device)
        self.meta = torch.zeros(4, dtype=torch.int32, device=device)
        self.c_struct = STATE(self.b_prev.data_ptr(), self.r_prev.data_ptr(), self.P.data_ptr(),
                              self.Q.data_ptr(), self.pq.data_ptr(), self.meta.data_ptr(), kcap)

    def basis(self):
        """Recycled directions (P, Q, pq), oldest first (synchronises)."""
        active, count, head, _ = [int(v) for v in self.meta.cpu()]
        slots = [(head - count + 1 + j) % self.kcap for j in range(count)]
        return self.P[active, slots], self.Q[active, slots], self.pq[active, slots]


class Fewha:
    """One operator / solver instance on the current CUDA device."""

    def __init__(self, geom, noise_w, precision="f64", tile=0, grid=0):
        import torch
        self._torch = torch
        if not torch.cuda.is_available():
            raise RuntimeError("libfewha needs a CUDA device")
        self.lib = load_library()
        self.precision = precision
        self._g = make_geometry(geom, noise_w, precision, tile, grid)
        h = C.c_void_p()
        st = self.lib.fewha_create(C.byref(self._g), C.byref(h))
        if st != 0:
            raise FewhaError(st, "fewha_create")
        self._h = h
        self.n = self.lib.fewha_n_unknowns(h)
        self.n_slopes = self.lib.fewha_n_slopes(h)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.dtype = torch.float64 if precision == "f64" else torch.float32
        self.slope_dtype = {"f64": torch.float64, "f32": torch.float32, "bf16s": torch.bfloat16}[precision]
        self.n_layers = len(geom.layers)

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fewha_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- host-side tables -------------------------------------------------
    def layer_spacing(self, l):
        return self.lib.fewha_layer_spacing(self._h, l)

    def prior(self):
        out = np.empty(self.n)
        self._check(self.lib.fewha_get_prior(self._h, out.ctypes.data_as(C.POINTER(C.c_double))), "get_prior")
        return out

    def set_noise(self, noise_w, refresh_precond=True):
        """New noise weights 1/sigma_g^2 (C_eta^{-1}); refresh_precond rebuilds J's data term."""
        w = np.ascontiguousarray(np.asarray(noise_w, dtype=np.float64))
        if w.shape != (len(self._g.gs[:self._g.n_gs]),):
            raise ValueError("one weight per guide star")
        self._check(self.lib.fewha_set_noise(self._h, w.ctypes.data_as(C.POINTER(C.c_double)),
                                              1 if refresh_precond else 0), "fewha_set_noise")

    def set_pt_bands(self, rows_large, rows_small):
        """P^T gather band heights (layer rows) on the largest / smaller layers."""
        self._check(self.lib.fewha_set_pt_bands(self._h, int(rows_large), int(rows_small)), "fewha_set_pt_bands")

    def launch_info(self):
        """Launch shape chosen at creation (fewha_get_launch_info) as a dict."""
        li = LAUNCH_INFO()
        self._check(self.lib.fewha_get_launch_info(self._h, C.byref(li)), "get_launch_info")
        return {k: getattr(li, k) for k, _ in LAUNCH_INFO._fields_}

    def precond(self):
        out = np.empty(self.n)
        self._check(self.lib.fewha_get_precond(self._h, out.ctypes.data_as(C.POINTER(C.c_double))),
                    "get_precond")
        return out

    def _check(self, st, what):
        if st != 0:
            raise FewhaError(st, what)

    def _vec(self, t, n, dtype, name, host_ok=False):
        """Pointer of a contiguous tensor of n elements: a CUDA tensor, or with
        host_ok a page-locked (pinned) CPU tensor, which the kernels read in
        place over the host link."""
        torch = self._torch
        on_host = host_ok and isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.is_pinned()
        if not isinstance(t, torch.Tensor) or (t.device.type != "cuda" and not on_host) or t.dtype != dtype:
            raise TypeError("%s must be a CUDA tensor%s of %s" % (name, " or a pinned CPU tensor" if host_ok else "",
                                                                 dtype))
        if t.numel() != n or not t.is_contiguous():
            raise ValueError("%s must be contiguous with %d elements" % (name, n))
        return C.c_void_p(t.data_ptr())

    # -- compute ------------------------------------------------------------
    def apply_op(self, x, out=None):
        """y = M x (Eq. M)."""
        y = out if out is not None else self._torch.empty(self.n, dtype=self.dtype, device=self.device)
        self._check(self.lib.fewha_apply_op(self._h, self._vec(x, self.n, self.dtype, "x"),
                                            self._vec(y, self.n, self.dtype, "y"),
                                            _stream_ptr(self._torch)), "fewha_apply_op")
        return y

    def apply_op_noalloc(self, x, out=None):
        """y = M x through fewha_apply_op_noalloc: the library allocates
        nothing (its intermediates live in a statically reserved device array
        shared by all calls).  `out` lets the caller bring its own output."""
        y = out if out is not None else self._torch.empty(self.n, dtype=self.dtype, device=self.device)
        self._check(self.lib.fewha_apply_op_noalloc(self._h, self._vec(x, self.n, self.dtype, "x"),
                                                    self._vec(y, self.n, self.dtype, "y"),
                                                    _stream_ptr(self._torch)), "fewha_apply_op_noalloc")
        return y

    def apply_op_multi(self, x, out=None):
        """Y[v] = M X[v] for the rows of a (nvec, ld) tensor, one launch per stage."""
        torch = self._torch
        if x.dim() != 2 or x.dtype != self.dtype or x.device.type != "cuda" or x.stride(1) != 1:
            raise TypeError("x must be a CUDA (nvec, ld) tensor of %s with unit inner stride" % self.dtype)
        y = out if out is not None else torch.empty((x.shape[0], self.n), dtype=self.dtype, device=self.device)
        self._check(self.lib.fewha_apply_op_multi(self._h, C.c_void_p(x.data_ptr()), x.stride(0),
                                                  C.c_void_p(y.data_ptr()), y.stride(0), x.shape[0],
                                                  _stream_ptr(torch)), "fewha_apply_op_multi")
        return y

    def rhs(self, s, out=None):
        """b = W^{-T} A^T C_eta^{-1} s."""
        b = out if out is not None else self._torch.empty(self.n, dtype=self.dtype, device=self.device)
        self._check(self.lib.fewha_rhs(self._h, self._vec(s, self.n_slopes, self.slope_dtype, "s", host_ok=True),
                                       self._vec(b, self.n, self.dtype, "b"), _stream_ptr(self._torch)),
                    "fewha_rhs")
        return b

    def new_state(self, kcap):
        return FewhaState(self._torch, self.n, kcap, self.dtype, self.device)

    # -- mirror side of Algorithm 3 (ground DM on the pupil nodes) ---------------
    @property
    def n_actuators(self):
        return self.lib.fewha_n_actuators(self._h)

    def new_mirror(self):
        return self._torch.zeros(self.n_actuators, dtype=self.dtype, device=self.device)

    def fit(self, c, out=None):
        """a~ = F W^{-1} c (fitting step)."""
        a = out if out is not None else self.new_mirror()
        self._check(self.lib.fewha_fit(self._h, self._vec(c, self.n, self.dtype, "c"),
                                       self._vec(a, self.n_actuators, self.dtype, "a"),
                                       _stream_ptr(self._torch)), "fewha_fit")
        return a

    def pol_slopes(self, s, a_prev, out=None):
        """s + Gamma a_prev for every guide star (pseudo-open-loop slopes)."""
        o = out if out is not None else self._torch.empty_like(s)
        self._check(self.lib.fewha_pol_slopes(self._h, self._vec(s, self.n_slopes, self.slope_dtype, "s"),
                                              self._vec(a_prev, self.n_actuators, self.dtype, "a_prev"),
                                              self._vec(o, self.n_slopes, self.slope_dtype, "out"),
                                              _stream_ptr(self._torch)), "fewha_pol_slopes")
        return o

    def control(self, closed, gain, a_im1, a_i, a_fit, out=None):
        """Gain control of Algorithm 3; returns the next mirror shape."""
        na = self.n_actuators
        o = out if out is not None else self.new_mirror()
        self._check(self.lib.fewha_control(self._h, 1 if closed else 0, float(gain),
                                           self._vec(a_im1, na, self.dtype, "a_im1"),
                                           self._vec(a_i, na, self.dtype, "a_i"),
                                           self._vec(a_fit, na, self.dtype, "a_fit"),
                                           self._vec(o, na, self.dtype, "out"), _stream_ptr(self._torch)),
                    "fewha_control")
        return o

    def new_stats(self):
        return self._torch.zeros(STATS_BYTES, dtype=self._torch.uint8, device=self.device)

    def solve(self, s, c, state, max_iter, rtol=0.0, augmented=True, recycle_all=False,
              persistent=True, stats=None, true_res_every=0, rhs_in_state=False, c_out=None):
        """One time step; c is updated in place.  Returns the device stats buffer.
        true_res_every = N > 0 replaces the residual by b - M c after every N-th
        iteration; rhs_in_state: the state already holds this step's
        right-hand side (after fewha_deflate_warm_start), s is not read.
        s: a CUDA tensor, or a pinned CPU tensor that the kernel reads in place.
        c_out: optional CUDA or pinned CPU tensor that the solve kernel also
        writes the solution into at the end of the step."""
        co = None if c_out is None else self._vec(c_out, self.n, self.dtype, "c_out", host_ok=True)
        o = OPTS(int(max_iter), float(rtol), 1 if augmented else 0,
                 RECYCLE_ALL if recycle_all else RECYCLE_LAST,
                 LAUNCH_PERSISTENT if persistent else LAUNCH_PHASES, int(true_res_every),
                 1 if rhs_in_state else 0, 0, co)
        stats = stats if stats is not None else self.new_stats()
        sp = None if (rhs_in_state and s is None) else self._vec(s, self.n_slopes, self.slope_dtype, "s",
                                                                 host_ok=True)
        self._check(self.lib.fewha_solve(self._h, sp,
                                         self._vec(c, self.n, self.dtype, "c"), C.byref(state.c_struct),
                                         C.byref(o), C.c_void_p(stats.data_ptr()),
                                         _stream_ptr(self._torch)), "fewha_solve")
        return stats

    def set_timeout(self, ns):
        """Time limit of the solver's device-side waits (ns)."""
        self._check(self.lib.fewha_set_timeout(self._h, int(ns)), "fewha_set_timeout")

    TRACE_TAGS = {1: "R1 wfs(rhs)", 2: "R2 gather(rhs)", 6: "R3a fdwt fine(rhs)", 3: "R3b b,r0,P^T r0",
                  5: "init",
                  10: "UA1 update+idwt", 16: "A2 idwt fine", 12: "B wfs", 13: "C gather",
                  14: "D1 fdwt fine", 15: "D2E fdwt+axpy", 20: "TU idwt(c)", 21: "TA2 idwt fine",
                  22: "TB wfs", 23: "TC gather", 24: "TD1 fdwt fine", 25: "TE b-Mc"}

    def set_trace(self, buf):
        """Enables the phase trace into a CUDA uint64/int64 tensor of shape (cap, 4), or None."""
        if buf is None:
            self._check(self.lib.fewha_set_trace(self._h, None, 0), "fewha_set_trace")
            self._trace = None
            return
        self._check(self.lib.fewha_set_trace(self._h, C.c_void_p(buf.data_ptr()), buf.shape[0]),
                    "fewha_set_trace")
        self._trace = buf

    def read_trace(self):
        """Per-phase (tag, span_ns, barrier_ns, max_cta_ns) of the last traced solve
        (synchronises): span from CTA 0 leaving the previous barrier to the last
        CTA arriving, barrier wait after that, and the longest single-CTA phase."""
        t = self._trace.cpu().numpy().astype("int64")
        out = []
        prev = None
        for i in range(t.shape[0]):
            maxcta, end, passed, tag = t[i, 0], t[i, 1], t[i, 2], t[i, 3]
            if passed == 0:
                break
            span = int(end - prev) if prev is not None else 0
            out.append((self.TRACE_TAGS.get(int(tag), str(tag)), span, int(passed - end), int(maxcta)))
            prev = passed
        return out

    def store(self, src, dst):
        """dst <- src by a library kernel (fewha_store): e.g. a solution into a
        pinned CPU tensor without a copy-engine transfer on the stream.  Both
        contiguous, the same number of bytes (a multiple of 16)."""
        torch = self._torch
        for t, nm in ((src, "src"), (dst, "dst")):
            if not isinstance(t, torch.Tensor) or not t.is_contiguous() or not (
                    t.device.type == "cuda" or (t.device.type == "cpu" and t.is_pinned())):
                raise TypeError("%s must be a contiguous CUDA tensor or pinned CPU tensor" % nm)
        nb = src.numel() * src.element_size()
        if dst.numel() * dst.element_size() != nb:
            raise ValueError("src and dst differ in size")
        self._check(self.lib.fewha_store(C.c_void_p(dst.data_ptr()), C.c_void_p(src.data_ptr()), nb,
                                         _stream_ptr(torch)), "fewha_store")
        return dst

    @staticmethod
    def read_stats(stats):
        """Host copy of a stats buffer as a dict (synchronises)."""
        raw = bytes(stats.cpu().numpy().tobytes())
        st = STATS.from_buffer_copy(raw)
        return {"status": st.status, "iterations": st.iterations, "rel_res": st.rel_res,
                "bnorm": st.bnorm, "rz": st.rz, "basis_count": st.basis_count}


class MCAO_DESC(C.Structure):
    _fields_ = [("n_dm", C.c_int), ("dm_n", C.c_int * 4), ("dm_pitch", C.c_double * 4), ("dm_h", C.c_double * 4),
                ("n_dir", C.c_int), ("dir_x", C.c_double * 16), ("dir_y", C.c_double * 16)]


class McaoFit:
    """MCAO fitting onto several mirrors (fewha_mcao_*): `dms` is a list of
    (actuators per side, pitch [m], altitude [m]), `dirs` a list of fitting
    directions (theta_x, theta_y) [rad].  fit(c, a, iters) runs `iters` CG
    iterations on the normal equations from the start in `a` (overwritten)."""

    def __init__(self, fewha, dms, dirs):
        if not 1 <= len(dms) <= 4 or not 1 <= len(dirs) <= 16:
            raise ValueError("1..4 mirrors and 1..16 directions")
        self.f, self.lib = fewha, fewha.lib
        d = MCAO_DESC()
        d.n_dm = len(dms)
        for i, (n, pitch, h) in enumerate(dms):
            d.dm_n[i], d.dm_pitch[i], d.dm_h[i] = int(n), float(pitch), float(h)
        d.n_dir = len(dirs)
        for i, (tx, ty) in enumerate(dirs):
            d.dir_x[i], d.dir_y[i] = float(tx), float(ty)
        h = C.c_void_p()
        fewha._check(self.lib.fewha_mcao_create(fewha._h, C.byref(d), C.byref(h)), "fewha_mcao_create")
        self._h = h
        self.n_actuators = self.lib.fewha_mcao_n_actuators(h)

    def new_mirrors(self):
        return self.f._torch.zeros(self.n_actuators, dtype=self.f.dtype, device=self.f.device)

    def fit(self, c, a, iters=4):
        f = self.f
        f._check(self.lib.fewha_mcao_fit(self._h, f._vec(c, f.n, f.dtype, "c"),
                                         f._vec(a, self.n_actuators, f.dtype, "a"), int(iters),
                                         _stream_ptr(f._torch)), "fewha_mcao_fit")
        return a

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fewha_mcao_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FewhaBatch:
    """Many instances (Fewha handles of one precision) solved by one
    cooperative launch, each by its own group of CTAs (fewha_batch_*)."""

    def __init__(self, fewhas, ctas=None, rounds=None, tiles=None):
        import torch
        self._torch = torch
        self.fewhas = list(fewhas)
        self.lib = load_library()
        n = len(self.fewhas)
        hs = (C.c_void_p * n)(*[f._h.value for f in self.fewhas])
        cs = (C.c_int * n)(*ctas) if ctas is not None else None
        rs = (C.c_int * n)(*rounds) if rounds is not None else None
        ts = (C.c_int * (2 * n))(*[v for t in tiles for v in (t or (0, 0))]) if tiles is not None else None
        self.rounds = list(rounds) if rounds is not None else [0] * n
        b = C.c_void_p()
        st = self.lib.fewha_batch_create_ex(hs, n, cs, rs, ts, C.byref(b))
        if st != 0:
            raise FewhaError(st, "fewha_batch_create_ex")
        self._b = b
        self.n = n
        self.device = self.fewhas[0].device

    def ctas(self):
        out = (C.c_int * self.n)()
        self.lib.fewha_batch_ctas(self._b, out)
        return list(out)

    def tiles(self):
        out = (C.c_int * (2 * self.n))()
        self.lib.fewha_batch_tiles(self._b, out)
        return [(out[2 * i], out[2 * i + 1]) for i in range(self.n)]

    def new_stats(self):
        return self._torch.zeros(self.n * STATS_BYTES, dtype=self._torch.uint8, device=self.device)

    def solve(self, slopes, cs, states, max_iter, rtol=0.0, augmented=True, recycle_all=False, stats=None,
              true_res_every=0):
        """One time step of every instance; cs are updated in place."""
        n = self.n
        for f, sl, c in zip(self.fewhas, slopes, cs):
            f._vec(sl, f.n_slopes, f.slope_dtype, "s")
            f._vec(c, f.n, f.dtype, "c")
        sp = (C.c_void_p * n)(*[t.data_ptr() for t in slopes])
        cp = (C.c_void_p * n)(*[t.data_ptr() for t in cs])
        stt = (STATE * n)(*[s_.c_struct for s_ in states])
        o = OPTS(int(max_iter), float(rtol), 1 if augmented else 0, RECYCLE_ALL if recycle_all else RECYCLE_LAST,
                 LAUNCH_PERSISTENT, int(true_res_every))
        stats = stats if stats is not None else self.new_stats()
        st = self.lib.fewha_batch_solve(self._b, sp, cp, stt, C.byref(o), C.c_void_p(stats.data_ptr()),
                                        _stream_ptr(self._torch))
        if st != 0:
            raise FewhaError(st, "fewha_batch_solve")
        return stats

    def bind(self, slopes, cs, states, max_iter, rtol=0.0, augmented=True, recycle_all=False, stats=None,
             true_res_every=0):
        """Fixes the buffers of launch(): every launch solves one time step of every
        instance from the current contents of `slopes` into `cs` (fewha_batch_bind)."""
        n = self.n
        for f, sl, c in zip(self.fewhas, slopes, cs):
            f._vec(sl, f.n_slopes, f.slope_dtype, "s")
            f._vec(c, f.n, f.dtype, "c")
        sp = (C.c_void_p * n)(*[t.data_ptr() for t in slopes])
        cp = (C.c_void_p * n)(*[t.data_ptr() for t in cs])
        stt = (STATE * n)(*[s_.c_struct for s_ in states])
        o = OPTS(int(max_iter), float(rtol), 1 if augmented else 0, RECYCLE_ALL if recycle_all else RECYCLE_LAST,
                 LAUNCH_PERSISTENT, int(true_res_every))
        self._bound = (slopes, cs, states, stats if stats is not None else self.new_stats())
        st = self.lib.fewha_batch_bind(self._b, sp, cp, stt, C.byref(o), C.c_void_p(self._bound[3].data_ptr()))
        if st != 0:
            raise FewhaError(st, "fewha_batch_bind")
        return self._bound[3]

    def launch(self):
        """One time step over the bound buffers (no host work; capturable)."""
        st = self.lib.fewha_batch_launch(self._b, _stream_ptr(self._torch))
        if st != 0:
            raise FewhaError(st, "fewha_batch_launch")

    def capture_graph(self):
        """A CUDA graph of one launch() (replay() after writing the bound slopes)."""
        torch = self._torch
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.launch()
        torch.cuda.current_stream().wait_stream(s)
        return g

    def read_stats(self, stats):
        raw = stats.cpu().numpy().tobytes()
        out = []
        for i in range(self.n):
            stt = STATS.from_buffer_copy(raw[i * STATS_BYTES:(i + 1) * STATS_BYTES])
            out.append({"status": stt.status, "iterations": stt.iterations, "rel_res": stt.rel_res,
                        "bnorm": stt.bnorm, "basis_count": stt.basis_count})
        return out

    def close(self):
        if getattr(self, "_b", None):
            self.lib.fewha_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _split(cap, work):
    """CTAs for instances of the given work filling `cap` CTAs in proportion
    to work, at least one each (cap >= number of instances)."""
    tot = float(sum(work))
    c = [max(1, int(cap * w / tot)) for w in work]
    while sum(c) > cap:
        c[max(range(len(c)), key=lambda i: c[i])] -= 1
    while sum(c) < cap:
        c[max(range(len(c)), key=lambda i: work[i] / c[i])] += 1
    return c


def _time_batch(batch, step, reps):
    """ms per batched time step of `step(batch)` over reps steps (after one)."""
    import torch
    step(batch)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        step(batch)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune_batch(fewhas, step, candidates=None, reps=3, tiles=((8, 8), (16, 16), (16, 24), (24, 24),
                                                                   (32, 32)),
                   bands=((8, 4), (4, 4), (8, 8), (4, 2), (2, 2)), log=None):
    """Chooses the launch shape of a batch by timing `step(batch)` (one
    batched time step).  Instances with the same geometry (unknowns, guide
    stars, subapertures) form a class and share their settings.  Stages:
      1. CTA split and rounds: the library's work-proportional split in one
         round; two rounds with the largest class first on the whole GPU
         (CTAs per instance = SMs / instances of that class, in one or in two
         rounds of its own) and the others after it, split in proportion to
         their work.  `candidates` (a list of (ctas, rounds) pairs) replaces
         the generated ones.
      2. WFS tile shape per class (`tiles`), in turn, keeping a change only
         when the step gets faster.
      3. P^T band heights per class (`bands`: rows on the largest and on the
         smaller layers of the geometry), the same way (set on the handles).
    The CTA cap is the device's SM count (one CTA of 512 threads per SM).
    Returns ({"ctas", "rounds", "tiles", "bands", "ms"}, timings): the best
    setting (the handles keep its band heights) and every timed candidate."""
    import torch
    n = len(fewhas)
    cap = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    say = log or (lambda *a: None)
    key = [(f.n, f.n_slopes) for f in fewhas]
    classes = sorted(set(key), key=lambda k: -k[0])
    members = {k: [i for i in range(n) if key[i] == k] for k in classes}
    timings = []

    def run(ctas, rounds, tl):
        try:
            b = FewhaBatch(fewhas, ctas, rounds, tl)
        except FewhaError:
            timings.append(((ctas, rounds, tl), None))
            return None, None
        ms = _time_batch(b, step, reps)
        got = (b.ctas(), list(b.rounds), b.tiles())
        b.close()
        timings.append((got, ms))
        say("autotune %s -> %.3f ms" % (got[0][:1] + got[0][-1:], ms))
        return ms, got

    # stage 1: CTA split and rounds
    if candidates is None:
        work = [f.n for f in fewhas]
        big = members[classes[0]]
        rest = [i for i in range(n) if i not in big]
        candidates = [(None, None)]
        if rest:
            # the largest class first on all SMs (in one or two rounds), the
            # others after it
            for parts in (1, 2):
                per = (len(big) + parts - 1) // parts
                c = [0] * n
                r = [0] * n
                for j, i in enumerate(big):
                    c[i] = max(1, cap // per)
                    r[i] = j // per
                for i, ci in zip(rest, _split(cap, [work[i] for i in rest])):
                    c[i] = ci
                    r[i] = parts
                candidates.append((c, r))
        else:
            candidates.append((_split(cap, [f.n for f in fewhas]), None))
    best_ms, best = float("inf"), None
    for ctas, rounds in candidates:
        ms, got = run(ctas, rounds, None)
        if ms is not None and ms < best_ms:
            best_ms, best = ms, got
    if best is None:
        raise FewhaError(-1, "autotune_batch: no candidate launch fits")
    ctas, rounds, tl = best
    # stage 2: WFS tiles per class
    for k in classes:
        for t in tiles:
            if all(tl[i] == t for i in members[k]):
                continue
            trial = [t if i in members[k] else tl[i] for i in range(n)]
            ms, got = run(ctas, rounds, trial)
            if ms is not None and ms < best_ms:
                best_ms, tl = ms, got[2]
    # stage 3: P^T band heights per class
    band = {}
    for k in classes:
        f0 = fewhas[members[k][0]]
        li = f0.launch_info()
        cur = (li["pt_rows_large"], li["pt_rows_small"])
        for bl in bands:
            if bl == cur:
                continue
            try:
                for i in members[k]:
                    fewhas[i].set_pt_bands(*bl)
            except FewhaError:
                continue
            ms, got = run(ctas, rounds, tl)
            if ms is not None and ms < best_ms:
                best_ms, cur = ms, bl
        for i in members[k]:
            fewhas[i].set_pt_bands(*cur)
        band[k] = cur
    return ({"ctas": ctas, "rounds": rounds, "tiles": tl, "bands": [band[key[i]] for i in range(n)],
             "ms": best_ms}, timings)

def read_bandwidth(nbytes, reps=20):
    """Read bandwidth [GB/s] of the library's streaming probe over a device
    buffer of nbytes (fewha_read_probe: one launch reading it reps times),
    timed with CUDA events after one untimed pass: an L2-resident buffer
    measures the L2, a large one DRAM."""
    import torch
    lib = load_library()
    buf = torch.ones(nbytes // 4, dtype=torch.float32, device="cuda")
    sink = torch.empty(4 * torch.cuda.get_device_properties(0).multi_processor_count, dtype=torch.float32,
                       device="cuda")
    stream = _stream_ptr(torch)
    st = lib.fewha_read_probe(C.c_void_p(buf.data_ptr()), buf.numel() * 4, 1, C.c_void_p(sink.data_ptr()), stream)
    if st != 0:
        raise FewhaError(st, "fewha_read_probe")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    lib.fewha_read_probe(C.c_void_p(buf.data_ptr()), buf.numel() * 4, reps, C.c_void_p(sink.data_ptr()), stream)
    e1.record()
    torch.cuda.synchronize()
    return buf.numel() * 4 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
