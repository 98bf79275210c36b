"""ctypes binding of libpeps_vmc.so (declarations: include/peps_vmc.h).

Argument marshalling only: every step of the cooling path runs in the CUDA library.
Importing works without a GPU; creating a context needs the built library and a GPU and
raises if either is missing (there is no CPU fallback).
"""
import ctypes
import os

import numpy as np

from .build import LIB

PEPS_OK = 0
PEPS_WARN_CG_MAXIT = 1
PEPS_EINVAL = -1
PEPS_ENOMEM = -2
PEPS_ECUDA = -3
PEPS_ESTATE = -4
PEPS_ENOTFINITE = -5
PEPS_ECORRUPT = -6
PEPS_EIO = -7
PEPS_ETIMEOUT = -8
PEPS_FP64 = 0
PEPS_FP32 = 1
PEPS_TF32 = 2
PEPS_MODEL_J1J2 = 0
PEPS_BLOCKS_AUTO = 0
PEPS_BLOCKS_NARROW = 1
PEPS_BLOCKS_WIDE = 2
PEPS_BLOCKS_BATCHED = 3

EXPORTS = [
    "peps_init", "peps_mc_sweep", "peps_eval_batch", "peps_sr_step", "peps_observables",
    "peps_step", "peps_get_theta", "peps_set_theta", "peps_get_configs", "peps_set_configs",
    "peps_num_params", "peps_o_row_len", "peps_sweeps_done", "peps_set_sweeps_done",
    "peps_last_counters", "peps_free", "peps_last_error", "peps_version", "peps_checkpoint",
    "peps_restore", "peps_time", "peps_eval_batch_noalloc", "peps_footprint",
    "peps_srv_create", "peps_srv_submit", "peps_srv_poll", "peps_srv_theta", "peps_srv_drain",
    "peps_srv_metrics", "peps_srv_free", "peps_launches", "peps_profile", "peps_profile_read",
    "peps_selftest_tc_timeout", "peps_autotune", "peps_profile_launch_bytes", "peps_set_tune", "peps_su_theta", "peps_su_warm_start", "peps_set_cg_product", "peps_srv_stop", "peps_cv_spline", "peps_set_graphs", "peps_graphs_captured",
    "peps_direct_draw", "peps_direct_next_bd", "peps_direct_step",
    "peps_group_create", "peps_group_eval", "peps_group_last_error", "peps_group_free",
    "peps_set_trunc_fp64", "peps_famp_create", "peps_famp_eval", "peps_famp_last_error",
    "peps_famp_free", "peps_famp_local_energy", "peps_famp_log_derivative",
    "peps_famp_n_moves", "peps_famp_sweep", "peps_famp_sr_step", "peps_famp_profile",
    "peps_famp_profile_read", "peps_famp_launches", "peps_famp_init_theta",
    "peps_famp_move_table", "peps_famp_set_strips",
]


class Params(ctypes.Structure):
    _fields_ = [("L1", ctypes.c_int), ("L2", ctypes.c_int), ("model", ctypes.c_int),
                ("J1", ctypes.c_double), ("J2", ctypes.c_double), ("D", ctypes.c_int),
                ("chi", ctypes.c_int), ("n_chains", ctypes.c_int), ("precision", ctypes.c_int),
                ("init_noise", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("n_blocks", ctypes.c_int), ("block_mode", ctypes.c_int)]


class Tune(ctypes.Structure):
    _fields_ = [("grid_pct", ctypes.c_int), ("db_bytes", ctypes.c_int), ("ffma_g", ctypes.c_int),
                ("kc_max", ctypes.c_int), ("ms_before", ctypes.c_double), ("ms_after", ctypes.c_double),
                ("pipelined", ctypes.c_int), ("stage_kb", ctypes.c_int),
                ("trunc_threads", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("beta_obs", ctypes.c_double), ("E_site", ctypes.c_double),
                ("E_err", ctypes.c_double), ("C_site", ctypes.c_double), ("chi_sus", ctypes.c_double),
                ("accept", ctypes.c_double), ("diag_frac", ctypes.c_double), ("cg_iters", ctypes.c_int),
                ("cg_resid", ctypes.c_double), ("p", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(ctypes.Structure):
    _fields_ = [("params", Params), ("tau", ctypes.c_double), ("t_end", ctypes.c_double),
                ("eps", ctypes.c_double), ("cg_tol", ctypes.c_double), ("max_cg", ctypes.c_int),
                ("n_sweeps", ctypes.c_int), ("n_burn", ctypes.c_int),
                ("p1_until_beta", ctypes.c_double)]


PEPS_REQ_QUEUED, PEPS_REQ_RUNNING, PEPS_REQ_DONE, PEPS_REQ_FAILED, PEPS_REQ_CANCELLED = 0, 1, 2, 3, 4

_lib = None


def load(path=None):
    """Loads the library (once).  Raises OSError when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise OSError(f"libpeps_vmc.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.peps_init.argtypes = [ctypes.POINTER(Params), vp, ctypes.POINTER(vp)]
    lib.peps_mc_sweep.argtypes = [vp, ip, ip]
    lib.peps_eval_batch.argtypes = [vp, vp, ip, ip, vp, vp, vp, vp, vp]
    lib.peps_sr_step.argtypes = [vp, dp, dp, ip, dp, ip, ctypes.POINTER(Stats)]
    lib.peps_observables.argtypes = [vp, ip, ctypes.POINTER(Stats)]
    lib.peps_step.argtypes = [vp, ip, ip, dp, dp, ip, dp, ctypes.POINTER(Stats)]
    lib.peps_get_theta.argtypes = [vp, vp, ctypes.c_size_t]
    lib.peps_set_theta.argtypes = [vp, vp, ctypes.c_size_t]
    lib.peps_get_configs.argtypes = [vp, vp, ctypes.c_size_t]
    lib.peps_set_configs.argtypes = [vp, vp, ctypes.c_size_t]
    lib.peps_num_params.argtypes = [vp]
    lib.peps_num_params.restype = ctypes.c_size_t
    lib.peps_o_row_len.argtypes = [vp]
    lib.peps_o_row_len.restype = ctypes.c_size_t
    lib.peps_sweeps_done.argtypes = [vp]
    lib.peps_sweeps_done.restype = ctypes.c_int64
    lib.peps_set_sweeps_done.argtypes = [vp, ctypes.c_int64]
    lib.peps_last_counters.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64)]
    lib.peps_checkpoint.argtypes = [vp, ctypes.c_char_p]
    lib.peps_restore.argtypes = [vp, ctypes.c_char_p]
    lib.peps_time.argtypes = [vp]
    lib.peps_time.restype = ctypes.c_double
    lib.peps_eval_batch_noalloc.argtypes = [ctypes.POINTER(Params), vp, vp, ip, vp, vp, vp, vp,
                                            vp, vp]
    lib.peps_footprint.argtypes = [ctypes.POINTER(Params)]
    lib.peps_footprint.restype = ctypes.c_size_t
    lib.peps_srv_create.argtypes = [ctypes.c_size_t, ip, ip, ctypes.POINTER(vp)]
    lib.peps_srv_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ip)]
    lib.peps_srv_poll.argtypes = [vp, ip, ctypes.POINTER(ip), ctypes.POINTER(ip),
                                  ctypes.POINTER(Stats), ip]
    lib.peps_srv_theta.argtypes = [vp, ip, vp, ctypes.c_size_t]
    lib.peps_srv_drain.argtypes = [vp]
    lib.peps_srv_stop.argtypes = [vp]
    lib.peps_srv_metrics.argtypes = [vp, ctypes.POINTER(dp), ctypes.POINTER(dp),
                                     ctypes.POINTER(dp), ctypes.POINTER(ctypes.c_int64)]
    lib.peps_srv_free.argtypes = [vp]
    lib.peps_srv_free.restype = None
    lib.peps_free.argtypes = [vp]
    lib.peps_free.restype = None
    lib.peps_last_error.argtypes = [vp]
    lib.peps_last_error.restype = ctypes.c_char_p
    lib.peps_version.restype = ctypes.c_char_p
    lib.peps_selftest_tc_timeout.argtypes = []
    lib.peps_autotune.argtypes = [vp, ip, ctypes.POINTER(Tune)]
    lib.peps_launches.argtypes = [vp]
    lib.peps_launches.restype = ctypes.c_longlong
    lib.peps_profile.argtypes = [vp, ip]
    lib.peps_profile_read.argtypes = [vp, ctypes.POINTER(KernelStat), ip, ctypes.POINTER(ip)]
    lib.peps_set_tune.argtypes = [vp, ctypes.POINTER(Tune)]
    lib.peps_su_warm_start.argtypes = [vp, dp, ip]
    lib.peps_set_cg_product.argtypes = [vp, ip]
    lib.peps_set_trunc_fp64.argtypes = [vp, ip]
    lib.peps_famp_create.argtypes = [ip, ip, ip, ip, ip, ip, vp, ctypes.POINTER(vp)]
    lib.peps_famp_eval.argtypes = [vp, vp, ctypes.c_size_t, vp, ip, vp, vp]
    lib.peps_famp_local_energy.argtypes = [vp, vp, ctypes.c_size_t, vp, ip, dp, dp, dp, vp, vp, vp, vp]
    lib.peps_famp_log_derivative.argtypes = [vp, vp, ctypes.c_size_t, vp, ip, vp]
    lib.peps_famp_n_moves.argtypes = [vp]
    lib.peps_famp_profile.argtypes = [vp, ip]
    lib.peps_famp_profile_read.argtypes = [vp, vp, ip, vp]
    lib.peps_famp_launches.argtypes = [vp]
    lib.peps_famp_launches.restype = ctypes.c_longlong
    lib.peps_famp_init_theta.argtypes = [ip, ip, ip, dp, ctypes.c_uint64, vp, ctypes.c_size_t]
    lib.peps_famp_move_table.argtypes = [ip, ip, vp, ip]
    lib.peps_famp_set_strips.argtypes = [vp, ip]
    lib.peps_famp_sweep.argtypes = [vp, vp, ctypes.c_size_t, vp, ip, ip, ip, ctypes.c_uint64,
                                    ctypes.c_uint64, vp, vp, vp, vp]
    lib.peps_famp_sr_step.argtypes = [vp, vp, ctypes.c_size_t, vp, ip, dp, dp, dp, ip, dp, dp, ip,
                                      dp, vp]
    lib.peps_famp_last_error.argtypes = [vp]
    lib.peps_famp_last_error.restype = ctypes.c_char_p
    lib.peps_famp_free.argtypes = [vp]
    lib.peps_famp_free.restype = None
    lib.peps_set_graphs.argtypes = [vp, ip]
    lib.peps_graphs_captured.argtypes = [vp]
    lib.peps_cv_spline.argtypes = [vp, vp, ip, dp, vp, vp, ip]
    lib.peps_direct_draw.argtypes = [vp, vp, ip, dp, dp, vp]
    lib.peps_group_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp)]
    lib.peps_group_eval.argtypes = [vp]
    lib.peps_group_last_error.argtypes = [vp]
    lib.peps_group_last_error.restype = ctypes.c_char_p
    lib.peps_group_free.argtypes = [vp]
    lib.peps_group_free.restype = None
    lib.peps_direct_next_bd.argtypes = [dp, dp, ip]
    lib.peps_direct_next_bd.restype = ctypes.c_double
    lib.peps_direct_step.argtypes = [vp, ctypes.POINTER(ctypes.c_double), dp, dp, dp, ip, dp,
                                     ctypes.POINTER(Stats)]
    lib.peps_su_theta.argtypes = [ip, ip, ip, dp, dp, ip, ctypes.POINTER(ctypes.c_double),
                                  ctypes.c_size_t]
    lib.peps_profile_launch_bytes.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                              ip, ctypes.POINTER(ip)]
    _lib = lib
    return lib


class PepsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"peps error {code}: {msg}")
        self.code = code


def su_theta(L1, L2, D, J1, tau, n_steps):
    """Parameters after the library's simple-update warm start (peps_su_theta: host-side,
    no GPU); hand them to Context.set_theta for SR from t = n_steps * tau."""
    lib = load()
    n = 0
    for r in range(L1):
        for c in range(L2):
            n += 4 * (1 if c == 0 else D) * (1 if c == L2 - 1 else D) * (1 if r == 0 else D) * \
                (1 if r == L1 - 1 else D)
    out = np.zeros(n)
    rc = lib.peps_su_theta(L1, L2, D, J1, tau, n_steps,
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n)
    if rc != PEPS_OK:
        raise PepsError(rc, "su_theta: invalid arguments")
    return out


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def cv_spline(betas, E_site, beta_eval, smoothing=0.0):
    """C/N = -beta^2 dE/dbeta from a natural cubic smoothing spline through (betas, E_site)
    (peps_cv_spline; smoothing bounds the residual sum of squares, 0 interpolates)."""
    b = np.ascontiguousarray(betas, dtype=np.float64)
    e = np.ascontiguousarray(E_site, dtype=np.float64)
    q = np.ascontiguousarray(np.atleast_1d(beta_eval), dtype=np.float64)
    out = np.empty(q.size, np.float64)
    rc = load().peps_cv_spline(_ptr(b), _ptr(e), int(b.size), float(smoothing), _ptr(q), _ptr(out),
                               int(q.size))
    if rc != PEPS_OK:
        raise PepsError(rc, "peps_cv_spline failed")
    return out


class Context:
    """One cooling run: PEPS parameters, Markov chains and work buffers on the GPU."""

    def __init__(self, L1, L2, D, chi, n_chains, J1=1.0, J2=0.0, precision=PEPS_FP64,
                 init_noise=1e-3, seed=0, n_blocks=0, stream=None, block_mode=PEPS_BLOCKS_AUTO):
        self.lib = load()
        self.params = Params(L1=L1, L2=L2, model=PEPS_MODEL_J1J2, J1=J1, J2=J2, D=D, chi=chi,
                             n_chains=n_chains, precision=precision, init_noise=init_noise,
                             seed=seed, n_blocks=n_blocks, block_mode=block_mode)
        self.ctx = ctypes.c_void_p()
        rc = self.lib.peps_init(ctypes.byref(self.params), stream, ctypes.byref(self.ctx))
        if rc != PEPS_OK:
            raise PepsError(rc, "peps_init failed")
        self.L1, self.L2, self.N = L1, L2, L1 * L2
        self.n_chains = n_chains
        self.precision = precision
        self.Np = int(self.lib.peps_num_params(self.ctx))
        self.No = int(self.lib.peps_o_row_len(self.ctx))
        self.o_dtype = np.float64 if precision == PEPS_FP64 else np.float32

    def _check(self, rc, allow=(PEPS_OK,)):
        if rc not in allow:
            raise PepsError(rc, self.lib.peps_last_error(self.ctx).decode())
        return rc

    def autotune(self, reps=1):
        """Tunes the batched engine's launch shapes on this context's chains (results are
        unchanged); reps=0 reports the current choice."""
        t = Tune()
        self._check(self.lib.peps_autotune(self.ctx, reps, ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in Tune._fields_}

    def set_tune(self, grid_pct, db_bytes, ffma_g, kc_max, pipelined=1, stage_kb=0, trunc_threads=0):
        """Pins the batched engine's launch shapes (results are unchanged); stage_kb=0 and
        trunc_threads=0 keep those two as they are."""
        t = Tune(grid_pct=grid_pct, db_bytes=db_bytes, ffma_g=ffma_g, kc_max=kc_max,
                 pipelined=pipelined, stage_kb=stage_kb, trunc_threads=trunc_threads)
        self._check(self.lib.peps_set_tune(self.ctx, ctypes.byref(t)))

    def launches(self):
        """Kernel launches this context has made so far."""
        return int(self.lib.peps_launches(self.ctx))

    def profile(self, enable, gemm_only=False):
        """Starts (True: cleared) or stops per-kernel event timing of this context; with
        gemm_only, only the batched GEMM kernels are timed."""
        self._check(self.lib.peps_profile(self.ctx, (2 if gemm_only else 1) if enable else 0))

    def profile_read(self):
        """Per-kernel {name: (launches, ms, bytes, flops)} since profiling started."""
        cap = 64
        buf = (KernelStat * cap)()
        n = ctypes.c_int()
        self._check(self.lib.peps_profile_read(self.ctx, buf, cap, ctypes.byref(n)))
        return {buf[i].name.decode(): (buf[i].launches, buf[i].ms, buf[i].bytes, buf[i].flops)
                for i in range(min(cap, n.value))}

    def profile_launch_bytes(self, name, cap=1 << 16):
        """Algorithmic bytes of each recorded launch of kernel `name` (not yet folded by
        profile_read), in launch order."""
        buf = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        self._check(self.lib.peps_profile_launch_bytes(self.ctx, name.encode(), buf, cap,
                                                       ctypes.byref(n)))
        return [buf[i] for i in range(min(cap, n.value))]

    def close(self):
        if self.ctx:
            self.lib.peps_free(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state
    def get_theta(self):
        out = np.empty(self.Np, np.float64)
        self._check(self.lib.peps_get_theta(self.ctx, _ptr(out), self.Np))
        return out

    def set_theta(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        self._check(self.lib.peps_set_theta(self.ctx, _ptr(th), th.size))

    def get_configs(self):
        out = np.empty((self.n_chains, self.N), np.uint8)
        self._check(self.lib.peps_get_configs(self.ctx, _ptr(out), out.size))
        return out

    def set_configs(self, S):
        S = np.ascontiguousarray(S, dtype=np.uint8)
        self._check(self.lib.peps_set_configs(self.ctx, _ptr(S), S.size))

    @property
    def t(self):
        return float(self.lib.peps_time(self.ctx))

    def checkpoint(self, path):
        self._check(self.lib.peps_checkpoint(self.ctx, str(path).encode()))

    def restore(self, path):
        self._check(self.lib.peps_restore(self.ctx, str(path).encode()))

    @property
    def sweeps_done(self):
        return int(self.lib.peps_sweeps_done(self.ctx))

    @sweeps_done.setter
    def sweeps_done(self, v):
        self._check(self.lib.peps_set_sweeps_done(self.ctx, int(v)))

    # -- the cooling path
    def mc_sweep(self, n_sweeps=1, p=2):
        self._check(self.lib.peps_mc_sweep(self.ctx, n_sweeps, p))

    def eval_batch(self, S=None, with_O=True):
        """Evaluates host configurations S (uint8 [nb][N]); S=None evaluates the chains.
        Returns numpy arrays (log_abs, sign, e_sys, e_anc, O or None)."""
        nb = self.n_chains if S is None else int(S.shape[0])
        la = np.empty(nb, np.float64)
        sg = np.empty(nb, np.int8)
        es = np.empty(nb, np.float64)
        ea = np.empty(nb, np.float64)
        O = np.empty((nb, self.No), self.o_dtype) if with_O else None
        Sp = None if S is None else _ptr(np.ascontiguousarray(S, dtype=np.uint8))
        self._check(self.lib.peps_eval_batch(self.ctx, Sp, nb, 0, _ptr(la), _ptr(sg), _ptr(es),
                                             _ptr(ea), _ptr(O)))
        return la, sg, es, ea, O

    def eval_batch_device(self, S, log_abs, sign, e_sys, e_anc, O=None):
        """Device-pointer variant (torch CUDA tensors)."""
        self._check(self.lib.peps_eval_batch(self.ctx, _ptr(S), int(S.shape[0]), 1, _ptr(log_abs),
                                             _ptr(sign), _ptr(e_sys), _ptr(e_anc), _ptr(O)))

    def eval_chains(self):
        """Evaluates the chains and keeps the results on the device for sr_step."""
        self._check(self.lib.peps_eval_batch(self.ctx, None, self.n_chains, 1, None, None, None,
                                             None, None))

    def sr_step(self, tau, eps=1e-4, max_cg=100, cg_tol=1e-10, p=2):
        st = Stats()
        rc = self._check(self.lib.peps_sr_step(self.ctx, tau, eps, max_cg, cg_tol, p,
                                               ctypes.byref(st)),
                         allow=(PEPS_OK, PEPS_WARN_CG_MAXIT))
        d = st.as_dict()
        d["cg_maxit"] = rc == PEPS_WARN_CG_MAXIT
        return d

    def observables(self, p=2):
        st = Stats()
        self._check(self.lib.peps_observables(self.ctx, p, ctypes.byref(st)))
        return st.as_dict()

    def step(self, n_sweeps=1, p=2, tau=0.02, eps=1e-4, max_cg=100, cg_tol=1e-10):
        st = Stats()
        rc = self._check(self.lib.peps_step(self.ctx, n_sweeps, p, tau, eps, max_cg, cg_tol,
                                            ctypes.byref(st)),
                         allow=(PEPS_OK, PEPS_WARN_CG_MAXIT))
        d = st.as_dict()
        d["cg_maxit"] = rc == PEPS_WARN_CG_MAXIT
        return d

    def direct_draw(self, u=None, b_d=1.0, exponent=0.5):
        """Replaces the chains by reweighted direct draws (peps_direct_draw) with host
        uniforms u (float64 [n_chains][N]) or, u=None, Philox uniforms.  Returns log q."""
        logq = np.empty(self.n_chains, np.float64)
        up = None
        if u is not None:
            u = np.ascontiguousarray(u, dtype=np.float64)
            if u.shape != (self.n_chains, self.N):
                raise ValueError("u must be [n_chains][L1*L2]")
            up = _ptr(u)
        self._check(self.lib.peps_direct_draw(self.ctx, up, 0, float(b_d), float(exponent),
                                              _ptr(logq)))
        return logq

    def direct_step(self, b_d, exponent=0.5, tau=0.02, eps=1e-4, max_cg=100, cg_tol=1e-10):
        """One cooling step on direct draws (peps_direct_step).  Returns (stats, next b_d)."""
        st = Stats()
        bd = ctypes.c_double(float(b_d))
        rc = self._check(self.lib.peps_direct_step(self.ctx, ctypes.byref(bd), float(exponent),
                                                   tau, eps, max_cg, cg_tol, ctypes.byref(st)),
                         allow=(PEPS_OK, PEPS_WARN_CG_MAXIT))
        d = st.as_dict()
        d["cg_maxit"] = rc == PEPS_WARN_CG_MAXIT
        return d, bd.value

    def set_graphs(self, on):
        """Captures and replays the batched engine's launch sequences (peps_set_graphs)."""
        self._check(self.lib.peps_set_graphs(self.ctx, 1 if on else 0))

    def graphs_captured(self):
        return int(self.lib.peps_graphs_captured(self.ctx))

    def set_trunc_fp64(self, on):
        """Float32 modes: Jacobi truncation on a float64 working copy (peps_set_trunc_fp64)."""
        self._check(self.lib.peps_set_trunc_fp64(self.ctx, 1 if on else 0))

    def set_cg_product(self, mode):
        """CG product form (peps_set_cg_product): 0 automatic, 1 fused single read, 2 two passes."""
        self._check(self.lib.peps_set_cg_product(self.ctx, int(mode)))

    def su_warm_start(self, tau, n_steps):
        """Simple-update warm start on the device (peps_su_warm_start): theta becomes the SU
        state at t = n_steps * tau and the context's time t with it."""
        self._check(self.lib.peps_su_warm_start(self.ctx, float(tau), int(n_steps)))

    def counters(self):
        f = ctypes.c_double()
        j = ctypes.c_int64()
        self._check(self.lib.peps_last_counters(self.ctx, ctypes.byref(f), ctypes.byref(j)))
        return f.value, j.value


class Group:
    """Several contexts whose chains are evaluated in one launch (peps_group_*): lattices of
    different sizes on the per-block engine's narrow blocks, one precision."""

    def __init__(self, contexts):
        self.lib = load()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.ctx.value for c in self.contexts])
        self.grp = ctypes.c_void_p()
        rc = self.lib.peps_group_create(arr, len(self.contexts), ctypes.byref(self.grp))
        if rc != PEPS_OK:
            raise PepsError(rc, "peps_group_create failed")

    def eval(self):
        """Evaluates every context's chains (kept on the device for sr_step/observables)."""
        rc = self.lib.peps_group_eval(self.grp)
        if rc != PEPS_OK:
            raise PepsError(rc, self.lib.peps_group_last_error(self.grp).decode())

    def close(self):
        if self.grp:
            self.lib.peps_group_free(self.grp)
            self.grp = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FStats(ctypes.Structure):
    _fields_ = [("E_site", ctypes.c_double), ("E_err", ctypes.c_double), ("docc", ctypes.c_double),
                ("density", ctypes.c_double), ("cg_iters", ctypes.c_int),
                ("cg_resid", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FermionAmplitudes:
    """Amplitudes of a fermionic PEPS of the doubled Hubbard lattice (peps_famp_*): sixteen
    local states per site, parity-even float64 parameters [16][dl][dr][du][dd] per site."""

    def __init__(self, L1, L2, D, chi, n_max, precision=PEPS_FP64, stream=None):
        self.lib = load()
        self.N = L1 * L2
        self.precision = precision
        self.No = sum((1 if c == 0 else D) * (1 if c == L2 - 1 else D) * (1 if r == 0 else D) *
                      (1 if r == L1 - 1 else D) for r in range(L1) for c in range(L2))
        self.h = ctypes.c_void_p()
        rc = self.lib.peps_famp_create(L1, L2, D, chi, n_max, precision, stream, ctypes.byref(self.h))
        if rc != PEPS_OK:
            raise PepsError(rc, "peps_famp_create failed")

    def eval(self, theta, S):
        """(log|psi|, sign) of the configurations S (uint8 [nb][N], entries 0..15)."""
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.uint8)
        nb = int(S.shape[0])
        la = np.empty(nb, np.float64)
        sg = np.empty(nb, np.int8)
        rc = self.lib.peps_famp_eval(self.h, _ptr(theta), theta.size, _ptr(S), nb, _ptr(la), _ptr(sg))
        if rc != PEPS_OK:
            raise PepsError(rc, self.lib.peps_famp_last_error(self.h).decode())
        return la, sg

    def log_derivative(self, theta, S):
        """O rows [nb][N_o] of the configurations S (peps_famp_log_derivative)."""
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.uint8)
        nb = int(S.shape[0])
        O = np.empty((nb, self.No), np.float64 if self.precision == PEPS_FP64 else np.float32)
        rc = self.lib.peps_famp_log_derivative(self.h, _ptr(theta), theta.size, _ptr(S), nb, _ptr(O))
        if rc != PEPS_OK:
            raise PepsError(rc, self.lib.peps_famp_last_error(self.h).decode())
        return O

    def local_energy(self, theta, S, t_hop, U, mu):
        """(log|psi|, sign, E_sys, E_anc) of the configurations S (peps_famp_local_energy)."""
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        S = np.ascontiguousarray(S, dtype=np.uint8)
        nb = int(S.shape[0])
        la = np.empty(nb, np.float64)
        sg = np.empty(nb, np.int8)
        es = np.empty(nb, np.float64)
        ea = np.empty(nb, np.float64)
        rc = self.lib.peps_famp_local_energy(self.h, _ptr(theta), theta.size, _ptr(S), nb, float(t_hop),
                                             float(U), float(mu), _ptr(la), _ptr(sg), _ptr(es), _ptr(ea))
        if rc != PEPS_OK:
            raise PepsError(rc, self.lib.peps_famp_last_error(self.h).decode())
        return la, sg, es, ea

    def profile(self, enable):
        """Starts (cleared) or stops per-kernel event timing of this evaluator's launches."""
        rc = self.lib.peps_famp_profile(self.h, 1 if enable else 0)
        if rc != PEPS_OK:
            raise PepsError(rc, self.lib.peps_famp_last_error(self.h).decode())

    def profile_read(self):
        """Per-kernel {name: (launches, ms, bytes, flops)} since profiling started."""
        cap = 64
        buf = (KernelStat * cap)()
        n = ctypes.c_int()
        rc = self.lib.peps_famp_profile_read(self.h, buf, cap, ctypes.byref(n))
        if rc != PEPS_OK:
            raise PepsError(rc, self.lib.peps_famp_last_error(self.h).decode())
        return {buf[i].name.decode(): (buf[i].launches, buf[i].ms, buf[i].bytes, buf[i].flops)
                for i in range(min(cap, n.value))}

    def launches(self):
        """Kernel launches this evaluator has made so far."""
        return int(self.lib.peps_famp_launches(self.h))

    def set_strips(self, enable):
        """Sweeps and local energies on cached strips (peps_famp_set_strips)."""
        rc = self.lib.peps_famp_set_strips(self.h, 1 if enable else 0)
        if rc != PEPS_OK:
            raise PepsError(rc, self.lib.peps_famp_last_error(self.h).decode())

    @property
    def n_moves(self):
        """Proposals in one Metropolis sweep (peps_famp_n_moves)."""
        return int(self.lib.peps_famp_n_moves(self.h))

    def sweep(self, theta, S, p=2, n_sweeps=1, seed=0, sweep0=0, u=None):
        """n_sweeps Metropolis sweeps of the chains S (peps_famp_sweep): returns (S, accepted
        per chain, log|psi|, sign) at the final configurations.  u: None (Philox) or
        [n_sweeps][nb][n_moves] uniforms."""
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        S = np.array(S, dtype=np.uint8, order="C", copy=True)
        nb = int(S.shape[0])
        acc = np.zeros(nb, np.int32)
        la = np.empty(nb, np.float64)
        sg = np.empty(nb, np.int8)
        up = None
        if u is not None:
            u = np.ascontiguousarray(u, dtype=np.float64)
            if u.size != n_sweeps * nb * self.n_moves:
                raise ValueError("u must hold n_sweeps x nb x n_moves uniforms")
            up = _ptr(u)
        rc = self.lib.peps_famp_sweep(self.h, _ptr(theta), theta.size, _ptr(S), nb, int(p),
                                      int(n_sweeps), int(seed), int(sweep0), up, _ptr(acc),
                                      _ptr(la), _ptr(sg))
        if rc != PEPS_OK:
            raise PepsError(rc, self.lib.peps_famp_last_error(self.h).decode())
        return S, acc, la, sg

    def sr_step(self, theta, S, t_hop, U, mu, p=2, tau=0.02, eps=1e-4, max_cg=100, cg_tol=1e-10):
        """One SR step on the configurations S (peps_famp_sr_step): returns (theta', stats)."""
        th = np.array(theta, dtype=np.float64, order="C", copy=True)
        S = np.ascontiguousarray(S, dtype=np.uint8)
        st = FStats()
        rc = self.lib.peps_famp_sr_step(self.h, _ptr(th), th.size, _ptr(S), int(S.shape[0]),
                                        float(t_hop), float(U), float(mu), int(p), float(tau),
                                        float(eps), int(max_cg), float(cg_tol), ctypes.byref(st))
        if rc not in (PEPS_OK, PEPS_WARN_CG_MAXIT):
            raise PepsError(rc, self.lib.peps_famp_last_error(self.h).decode())
        d = st.as_dict()
        d["cg_maxit"] = rc == PEPS_WARN_CG_MAXIT
        return th, d

    def close(self):
        if self.h:
            self.lib.peps_famp_free(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def famp_init_theta(L1, L2, D, noise=1e-3, seed=0):
    """The infinite-temperature state |I> as fermionic PEPS parameters with parity-even Philox
    noise (peps_famp_init_theta)."""
    from .workloads import site_dims
    n = 16 * sum(int(np.prod(d)) for d in site_dims(L1, L2, D))
    th = np.empty(n, np.float64)
    rc = load().peps_famp_init_theta(int(L1), int(L2), int(D), float(noise), int(seed), _ptr(th), n)
    if rc != PEPS_OK:
        raise PepsError(rc, "peps_famp_init_theta failed")
    return th


def famp_move_table(L1, L2):
    """The moves of one fermionic sweep, [n_moves][4] (kind, i, j, spin or mode)
    (peps_famp_move_table)."""
    lib = load()
    n = lib.peps_famp_move_table(int(L1), int(L2), None, 0)
    if n < 0:
        raise PepsError(n, "peps_famp_move_table failed")
    t = np.empty((n, 4), np.int32)
    lib.peps_famp_move_table(int(L1), int(L2), _ptr(t), n)
    return t


def direct_next_bd(b_d, diag_frac, N):
    """The diagonal bias of the next direct draw (peps_direct_next_bd)."""
    return float(load().peps_direct_next_bd(float(b_d), float(diag_frac), int(N)))


class Server:
    """Continuous-batching serving loop of cooling runs (peps_srv_*)."""

    def __init__(self, hbm_budget=0, max_active=4, blocks_per_request=0):
        self.lib = load()
        self.srv = ctypes.c_void_p()
        rc = self.lib.peps_srv_create(hbm_budget, max_active, blocks_per_request,
                                      ctypes.byref(self.srv))
        if rc != PEPS_OK:
            raise PepsError(rc, "peps_srv_create failed")
        self.nparams = {}

    def submit(self, L1, L2, D, chi, n_chains, t_end, tau=0.02, J1=1.0, J2=0.0,
               precision=PEPS_FP64, seed=0, init_noise=1e-3, eps=1e-4, cg_tol=1e-10, max_cg=100,
               n_sweeps=1, n_burn=2, p1_until_beta=0.3):
        P = Params(L1=L1, L2=L2, model=PEPS_MODEL_J1J2, J1=J1, J2=J2, D=D, chi=chi,
                   n_chains=n_chains, precision=precision, init_noise=init_noise, seed=seed,
                   n_blocks=0, block_mode=PEPS_BLOCKS_AUTO)
        q = Request(params=P, tau=tau, t_end=t_end, eps=eps, cg_tol=cg_tol, max_cg=max_cg,
                    n_sweeps=n_sweeps, n_burn=n_burn, p1_until_beta=p1_until_beta)
        rid = ctypes.c_int()
        rc = self.lib.peps_srv_submit(self.srv, ctypes.byref(q), ctypes.byref(rid))
        if rc != PEPS_OK:
            raise PepsError(rc, "peps_srv_submit failed")
        from .workloads import n_params
        self.nparams[rid.value] = n_params(L1, L2, D)
        return rid.value

    def poll(self, rid, cap=4096):
        st, n = ctypes.c_int(), ctypes.c_int()
        buf = (Stats * cap)()
        rc = self.lib.peps_srv_poll(self.srv, rid, ctypes.byref(st), ctypes.byref(n), buf, cap)
        if rc != PEPS_OK:
            raise PepsError(rc, "peps_srv_poll failed")
        return st.value, [buf[i].as_dict() for i in range(min(n.value, cap))]

    def theta(self, rid):
        out = np.empty(self.nparams[rid], np.float64)
        rc = self.lib.peps_srv_theta(self.srv, rid, _ptr(out), out.size)
        if rc != PEPS_OK:
            raise PepsError(rc, "peps_srv_theta failed")
        return out

    def drain(self):
        rc = self.lib.peps_srv_drain(self.srv)
        if rc != PEPS_OK:
            raise PepsError(rc, "a request failed")

    def stop(self):
        """Cancels queued requests and ends running ones after their current step."""
        rc = self.lib.peps_srv_stop(self.srv)
        if rc != PEPS_OK:
            raise PepsError(rc, "peps_srv_stop failed")

    def metrics(self):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        self.lib.peps_srv_metrics(self.srv, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                  ctypes.byref(n))
        return {"p50_ms": a.value, "p99_ms": b.value, "samples_per_s": c.value, "steps": n.value}

    def close(self):
        if self.srv:
            self.lib.peps_srv_free(self.srv)
            self.srv = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
