"""Thin Python binding of libmorap.so (include/morap.h).

Argument marshalling only: every step of the method runs in the library
(CUDA kernels and its host C++).  The binding refuses to run without the
built library -- there is no Python or CPU fallback.

Names follow the C-ABI.  Arrays are numpy; host outputs are returned as
numpy arrays.  `stream` is a cudaStream_t as an int (e.g.
torch.cuda.current_stream().cuda_stream) or None for the default stream.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmorap.so")

OK, EINVAL, ENOMEM, ENOTCONV, ECUDA, EBUSY, ESTATE = range(7)
PREC_MIXED, PREC_FP64 = 0, 1
_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOTCONV", 4: "ECUDA", 5: "EBUSY", 6: "ESTATE"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class MorapError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"morap error {_NAMES.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("eps_vi", ctypes.c_double),
        ("eps_eval", ctypes.c_double),
        ("tau_policy", ctypes.c_double),
        ("max_sweeps", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("device", ctypes.c_int32),
        ("launch_mode", ctypes.c_int32),
        ("hbm_budget", ctypes.c_size_t),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
        ("sweep_variant_fp32", ctypes.c_int32),
        ("sweep_variant_fp64", ctypes.c_int32),
        ("skip_unchanged", ctypes.c_int32),
        ("polish", ctypes.c_int32),
        ("eval_block", ctypes.c_int32),
        ("in_place", ctypes.c_int32),
        ("item_warps_max", ctypes.c_int32),
        ("tail_items", ctypes.c_int32),
    ]


class Footprint(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("n_products", "n_states", "n_sa", "n_trans", "csr_bytes",
                                              "device_bytes", "h2d_bytes")]


class SolveStats(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_int32), ("fp32_sweeps", ctypes.c_int32), ("fp64_sweeps", ctypes.c_int32),
        ("eval_sweeps", ctypes.c_int32),
        ("updates_fp32", ctypes.c_int64), ("updates_fp64", ctypes.c_int64), ("updates_eval", ctypes.c_int64),
        ("bytes_fp32", ctypes.c_int64), ("bytes_fp64", ctypes.c_int64), ("bytes_eval", ctypes.c_int64),
        ("ms_fp32", ctypes.c_double), ("ms_fp64", ctypes.c_double), ("ms_finalise", ctypes.c_double),
        ("ms_eval", ctypes.c_double), ("ms_host", ctypes.c_double), ("ms_total", ctypes.c_double),
        ("pairs_not_converged", ctypes.c_int32), ("eval_pairs", ctypes.c_int32),
        ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64), ("kernel_launches", ctypes.c_int32),
        ("variant_fp32", ctypes.c_int32), ("variant_fp64", ctypes.c_int32), ("polish", ctypes.c_int32),
        ("ms_tune", ctypes.c_double),
        ("skipped_fp32", ctypes.c_int64), ("skipped_fp64", ctypes.c_int64), ("work_items", ctypes.c_int64),
        ("computed_fp32", ctypes.c_int64), ("computed_fp64", ctypes.c_int64), ("anchored_states", ctypes.c_int64),
        ("tail_sweeps_fp32", ctypes.c_int32), ("tail_sweeps_fp64", ctypes.c_int32),
    ]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_batch", ctypes.c_int32), ("n_workers", ctypes.c_int32),
                ("eps", ctypes.c_double), ("max_iter", ctypes.c_int32), ("merge_instances", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("mean_batch", ctypes.c_double), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("queries_per_s", ctypes.c_double), ("wall_s", ctypes.c_double), ("bytes_in_use", ctypes.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class PointResult(ctypes.Structure):
    _fields_ = [
        ("feasible", ctypes.c_int32), ("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
        ("status", ctypes.c_int32), ("distance", ctypes.c_double),
        ("t_up", ctypes.POINTER(ctypes.c_double)), ("t_down", ctypes.POINTER(ctypes.c_double)),
        ("w_hist", ctypes.POINTER(ctypes.c_double)), ("r_hist", ctypes.POINTER(ctypes.c_double)),
        ("lambda_", ctypes.POINTER(ctypes.c_double)), ("assign_hist", ctypes.POINTER(ctypes.c_int32)),
    ]


_lib = None
_P = ctypes.c_void_p
_I32P = ctypes.POINTER(ctypes.c_int32)
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)
_U8P = ctypes.POINTER(ctypes.c_uint8)

_SIGS = {
    "morap_config_default": (None, [ctypes.POINTER(Config)]),
    "morap_ctx_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "morap_ctx_destroy": (ctypes.c_int, [_P]),
    "morap_last_error": (ctypes.c_char_p, []),
    "morap_add_agent": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _I32P, _I32P, _I32P, _DP, _DP, _I32P,
                                       _I32P, _I32P]),
    "morap_add_task": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _I32P, _I32P, _U8P,
                                      _I32P]),
    "morap_build": (ctypes.c_int, [_P, _P, ctypes.POINTER(Footprint)]),
    "morap_rebuild": (ctypes.c_int, [_P, _P]),
    "morap_solve": (ctypes.c_int, [_P, ctypes.c_int32, _DP, _P, _DP, _DP, _DP, _I32P]),
    "morap_supporting_points": (ctypes.c_int, [_P, ctypes.c_int32, _DP, _P, _DP, _I32P, _DP]),
    "morap_last_solve_stats": (ctypes.c_int, [_P, ctypes.POINTER(SolveStats)]),
    "morap_solve_plain": (ctypes.c_int, [_P, ctypes.c_int32, _I32P, _DP, _P, _DP, _DP, _DP, _DP]),
    "morap_query": (ctypes.c_int, [_P, _DP, _DP, ctypes.c_double, ctypes.c_int32, _P, ctypes.POINTER(PointResult)]),
    "morap_verify": (ctypes.c_int, [_P, _DP, _DP, ctypes.c_double, ctypes.c_int32, _P, ctypes.POINTER(PointResult)]),
    "morap_assign_max": (ctypes.c_int, [ctypes.c_int32, _DP, _I32P]),
    "morap_assign_tasks": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _DP, _I32P]),
    "morap_select_pairs": (ctypes.c_int, [_P, ctypes.c_int32, _I32P, _I32P]),
    "morap_random_assignment": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _DP, _I32P, _DP]),
    "morap_evaluate": (ctypes.c_int, [_P, ctypes.c_int32, _I32P, _I32P, _P, _DP, _DP]),
    "morap_pareto_create": (ctypes.c_int, [ctypes.c_int32, _DP, _DP, ctypes.c_double, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "morap_pareto_create_mode": (ctypes.c_int, [ctypes.c_int32, _DP, _DP, ctypes.c_double, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.POINTER(ctypes.c_void_p)]),
    "morap_pareto_next": (ctypes.c_int, [_P, _DP, _I32P]),
    "morap_pareto_step": (ctypes.c_int, [_P, _DP, ctypes.c_int32]),
    "morap_pareto_result": (ctypes.c_int, [_P, ctypes.POINTER(PointResult)]),
    "morap_pareto_destroy": (None, [_P]),
    "morap_project_halfspaces": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _DP, _DP, _DP, _DP, _DP]),
    "morap_project_down_hull": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _DP, _DP, _DP, _DP]),
    "morap_task_preprocess": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _I32P, _U8P, _I32P,
                                             _U8P]),
    "morap_product_info": (ctypes.c_int, [_P, ctypes.c_int32, _I64P]),
    "morap_product_download": (ctypes.c_int, [_P, ctypes.c_int32, _I64P, _I64P, _I32P, _DP, _DP, _I32P]),
    "morap_last_policy": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _U8P, _DP]),
    "morap_server_config_default": (None, [ctypes.POINTER(ServerConfig)]),
    "morap_server_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32,
                                           ctypes.POINTER(ServerConfig), ctypes.POINTER(ctypes.c_void_p)]),
    "morap_server_destroy": (ctypes.c_int, [_P]),
    "morap_submit": (ctypes.c_int, [_P, ctypes.c_int32, _DP, ctypes.POINTER(ctypes.c_int64)]),
    "morap_poll": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(PointResult)]),
    "morap_server_wait": (ctypes.c_int, [_P, ctypes.c_double]),
    "morap_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ServerStats)]),
    "morap_barrier_selfcheck": (ctypes.c_int, [ctypes.c_int32, _I32P, _DP]),
    "morap_plain_vi_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P, _P, ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_int32, _P, _P, _P, _DP, _I32P]),
}


def lib():
    """Load libmorap.so.  Raises if it has not been built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise MorapError(ECUDA, f"{LIB_PATH} is missing: build it first (paper_2305_04397_gb300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    return sorted(_SIGS)


def _check(rc):
    if rc != OK:
        raise MorapError(rc, lib().morap_last_error().decode())
    return rc


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype)) if a is not None else None


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _stream(s):
    return ctypes.c_void_p(int(s)) if s else None


# ---------------------------------------------------------------- C-ABI


def morap_config_default():
    cfg = Config()
    lib().morap_config_default(ctypes.byref(cfg))
    return cfg


def morap_ctx_create(cfg=None):
    h = ctypes.c_void_p()
    _check(lib().morap_ctx_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h)))
    return h


def morap_ctx_destroy(ctx):
    return _check(lib().morap_ctx_destroy(ctx))


def morap_add_agent(ctx, n_states, s0, state_ptr, sa_ptr, succ, prob, cost, label_ptr, label_ap):
    out = ctypes.c_int32()
    arrs = [_arr(state_ptr, np.int32), _arr(sa_ptr, np.int32), _arr(succ, np.int32), _arr(prob, np.float64),
            _arr(cost, np.float64), _arr(label_ptr, np.int32), _arr(label_ap, np.int32)]
    _check(lib().morap_add_agent(ctx, int(n_states), int(s0), _ptr(arrs[0], ctypes.c_int32),
                                 _ptr(arrs[1], ctypes.c_int32), _ptr(arrs[2], ctypes.c_int32),
                                 _ptr(arrs[3], ctypes.c_double), _ptr(arrs[4], ctypes.c_double),
                                 _ptr(arrs[5], ctypes.c_int32), _ptr(arrs[6], ctypes.c_int32), ctypes.byref(out)))
    return out.value


def morap_add_task(ctx, n_locs, q0, n_ap, ap_ids, delta, accepting):
    out = ctypes.c_int32()
    a = _arr(ap_ids, np.int32)
    d = _arr(delta, np.int32)
    acc = _arr(accepting, np.uint8)
    _check(lib().morap_add_task(ctx, int(n_locs), int(q0), int(n_ap), _ptr(a, ctypes.c_int32),
                                _ptr(d, ctypes.c_int32), _ptr(acc, ctypes.c_uint8), ctypes.byref(out)))
    return out.value


def morap_build(ctx, stream=None):
    fp = Footprint()
    _check(lib().morap_build(ctx, _stream(stream), ctypes.byref(fp)))
    return {n: getattr(fp, n) for n, _ in fp._fields_}


def morap_rebuild(ctx, stream=None):
    return _check(lib().morap_rebuild(ctx, _stream(stream)))


def morap_select_pairs(ctx, agent, task):
    a = _arr(agent, np.int32)
    t = _arr(task, np.int32)
    if a.shape != t.shape:
        raise ValueError("agent and task lists differ in length")
    return _check(lib().morap_select_pairs(ctx, len(a), _ptr(a, ctypes.c_int32), _ptr(t, ctypes.c_int32)))


def morap_solve(ctx, W, n_agents, n_tasks, stream=None, evaluate=True, check=True, n_pairs=None):
    """c, r_cost, r_prob and status as [K][|I|][|J|] arrays, or [K][n_pairs]
    for a context restricted by morap_select_pairs."""
    W = _arr(np.atleast_2d(W), np.float64)
    K = W.shape[0]
    shape = (K, n_pairs) if n_pairs is not None else (K, n_agents, n_tasks)
    P = int(np.prod(shape[1:]))
    c = np.zeros(shape)
    rc = np.zeros_like(c) if evaluate else None
    rp = np.zeros_like(c) if evaluate else None
    st = np.zeros(shape, np.int32)
    code = lib().morap_solve(ctx, K, _ptr(W, ctypes.c_double), _stream(stream), _ptr(c, ctypes.c_double),
                             _ptr(rc, ctypes.c_double), _ptr(rp, ctypes.c_double), _ptr(st, ctypes.c_int32))
    if check and code != ENOTCONV:
        _check(code)
    assert c.size == K * P
    return {"c": c, "r_cost": rc, "r_prob": rp, "status": st, "code": code}


def morap_supporting_points(ctx, W, n_agents, n_tasks, stream=None, want_c=False, check=True):
    W = _arr(np.atleast_2d(W), np.float64)
    K = W.shape[0]
    r = np.zeros((K, n_agents + n_tasks))
    f = np.zeros((K, n_tasks), np.int32)
    c = np.zeros((K, n_agents, n_tasks)) if want_c else None
    code = lib().morap_supporting_points(ctx, K, _ptr(W, ctypes.c_double), _stream(stream), _ptr(r, ctypes.c_double),
                                         _ptr(f, ctypes.c_int32), _ptr(c, ctypes.c_double))
    if check and code != ENOTCONV:
        _check(code)
    return {"r": r, "assign": f, "c": c, "code": code}


def morap_last_solve_stats(ctx):
    st = SolveStats()
    _check(lib().morap_last_solve_stats(ctx, ctypes.byref(st)))
    return st.as_dict()


def morap_solve_plain(ctx, pair_product, pair_w, stream=None, evaluate=True):
    pp = _arr(pair_product, np.int32)
    pw = _arr(pair_w, np.float64).reshape(-1, 2)
    n = len(pp)
    c = np.zeros(n)
    rc = np.zeros(n) if evaluate else None
    rp = np.zeros(n) if evaluate else None
    stats = np.zeros(4)
    code = lib().morap_solve_plain(ctx, n, _ptr(pp, ctypes.c_int32), _ptr(pw, ctypes.c_double), _stream(stream),
                                   _ptr(c, ctypes.c_double), _ptr(rc, ctypes.c_double), _ptr(rp, ctypes.c_double),
                                   _ptr(stats, ctypes.c_double))
    if code != ENOTCONV:
        _check(code)
    return {"c": c, "r_cost": rc, "r_prob": rp, "sweeps_vi": stats[0], "sweeps_eval": stats[1],
            "updates": stats[2], "ms": stats[3], "code": code}


def morap_query(ctx, t, M=None, eps=1e-6, max_iter=64, stream=None, check=True, n_tasks=None, verify_only=False):
    """Algorithm 1 (morap_query), or with verify_only=True the
    verification-only loop (morap_verify): a yes/no answer for t."""
    t = _arr(t, np.float64)
    n = len(t)
    Mm = _arr(M, np.float64) if M is not None else None
    t_up = np.zeros(n)
    t_dn = np.zeros(n)
    wh = np.zeros((max_iter, n))
    rh = np.zeros((max_iter, n))
    res = PointResult()
    res.t_up = _ptr(t_up, ctypes.c_double)
    res.t_down = _ptr(t_dn, ctypes.c_double)
    res.w_hist = _ptr(wh, ctypes.c_double)
    res.r_hist = _ptr(rh, ctypes.c_double)
    lam = np.zeros(max_iter)
    n_tasks = n_tasks if n_tasks is not None else 0
    fh = np.zeros((max_iter, max(n_tasks, 1)), np.int32)
    res.lambda_ = _ptr(lam, ctypes.c_double)
    res.assign_hist = _ptr(fh, ctypes.c_int32) if n_tasks else None
    fn = lib().morap_verify if verify_only else lib().morap_query
    code = fn(ctx, _ptr(t, ctypes.c_double), _ptr(Mm, ctypes.c_double), float(eps), int(max_iter), _stream(stream),
              ctypes.byref(res))
    if check and code not in (OK, ENOTCONV):
        _check(code)
    it = res.iterations
    out = {"feasible": bool(res.feasible), "iterations": it, "converged": bool(res.converged),
           "distance": res.distance, "t_up": t_up, "t_down": t_dn, "w_hist": wh[:it], "r_hist": rh[:it],
           "lambda": lam[:it], "code": code}
    if n_tasks:
        out["assign_hist"] = fh[:it]
    return out


def random_assignment(lam, assign_hist, n_agents):
    """The synthesised random assignment (morap_random_assignment):
    P[i][j] = probability that agent i does task j."""
    lam = _arr(lam, np.float64)
    F = _arr(assign_hist, np.int32)
    F = F.reshape(len(lam), -1) if F.size else np.zeros((len(lam), 0), np.int32)
    n_tasks = F.shape[1]
    P = np.zeros((n_agents, n_tasks))
    _check(lib().morap_random_assignment(len(lam), int(n_agents), n_tasks, _ptr(lam, ctypes.c_double),
                                         _ptr(F, ctypes.c_int32), _ptr(P, ctypes.c_double)))
    return P


class Pareto:
    """Algorithm 1 fed one supporting point at a time (morap_pareto_*)."""

    def __init__(self, t, M=None, eps=1e-6, max_iter=64, verify_only=False):
        self.t = _arr(t, np.float64)
        self.n = len(self.t)
        self.max_iter = int(max_iter)
        Mm = _arr(M, np.float64) if M is not None else None
        h = ctypes.c_void_p()
        _check(lib().morap_pareto_create_mode(self.n, _ptr(self.t, ctypes.c_double), _ptr(Mm, ctypes.c_double),
                                              float(eps), self.max_iter, 1 if verify_only else 0,
                                              ctypes.byref(h)))
        self.h = h

    def next(self):
        """The direction w whose supporting point step() needs, or None once the loop stopped."""
        w = np.zeros(self.n)
        done = ctypes.c_int32()
        _check(lib().morap_pareto_next(self.h, _ptr(w, ctypes.c_double), ctypes.byref(done)))
        return None if done.value else w

    def step(self, r, solve_status=OK):
        r = _arr(r, np.float64)
        _check(lib().morap_pareto_step(self.h, _ptr(r, ctypes.c_double), int(solve_status)))

    def result(self):
        n, it = self.n, self.max_iter
        t_up, t_dn = np.zeros(n), np.zeros(n)
        wh, rh = np.zeros((it, n)), np.zeros((it, n))
        res = PointResult()
        res.t_up = _ptr(t_up, ctypes.c_double)
        res.t_down = _ptr(t_dn, ctypes.c_double)
        res.w_hist = _ptr(wh, ctypes.c_double)
        res.r_hist = _ptr(rh, ctypes.c_double)
        lam = np.zeros(it)
        res.lambda_ = _ptr(lam, ctypes.c_double)
        code = lib().morap_pareto_result(self.h, ctypes.byref(res))
        if code not in (OK, ENOTCONV):
            _check(code)
        k = res.iterations
        return {"feasible": bool(res.feasible), "iterations": k, "converged": bool(res.converged),
                "distance": res.distance, "t_up": t_up, "t_down": t_dn, "w_hist": wh[:k], "r_hist": rh[:k],
                "lambda": lam[:k], "code": code}

    def close(self):
        if self.h:
            lib().morap_pareto_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def morap_assign_tasks(c):
    """Algorithm 2's assignment for c[K][|I|][|J|]: [K][|J|] agent per task (-1 = none)."""
    c = _arr(np.asarray(c, np.float64).reshape((-1,) + np.shape(c)[-2:]), np.float64)
    K, nI, nJ = c.shape
    f = np.zeros((K, nJ), np.int32)
    _check(lib().morap_assign_tasks(nI, nJ, K, _ptr(c, ctypes.c_double), _ptr(f, ctypes.c_int32)))
    return f


def morap_evaluate(ctx, pair_product, pair_weight, stream=None, check=True):
    """Algorithm 4 for chosen (product, weight-index) pairs of the last solve on ctx."""
    pp = _arr(pair_product, np.int32)
    pw = _arr(pair_weight, np.int32)
    rc = np.zeros(len(pp))
    rp = np.zeros(len(pp))
    code = lib().morap_evaluate(ctx, len(pp), _ptr(pp, ctypes.c_int32), _ptr(pw, ctypes.c_int32), _stream(stream),
                                _ptr(rc, ctypes.c_double), _ptr(rp, ctypes.c_double))
    if check and code != ENOTCONV:
        _check(code)
    return {"r_cost": rc, "r_prob": rp, "code": code}


def morap_assign_max(C):
    C = _arr(C, np.float64)
    n = C.shape[0]
    f = np.zeros(n, np.int32)
    _check(lib().morap_assign_max(n, _ptr(C, ctypes.c_double), _ptr(f, ctypes.c_int32)))
    return f


def morap_project_halfspaces(t, A, b, M=None):
    t = _arr(t, np.float64)
    A = _arr(np.atleast_2d(A), np.float64)
    b = _arr(b, np.float64)
    z = np.zeros(len(t))
    Mm = _arr(M, np.float64) if M is not None else None
    _check(lib().morap_project_halfspaces(len(t), A.shape[0], _ptr(t, ctypes.c_double), _ptr(A, ctypes.c_double),
                                          _ptr(b, ctypes.c_double), _ptr(Mm, ctypes.c_double),
                                          _ptr(z, ctypes.c_double)))
    return z


def morap_project_down_hull(t, Phi, M=None):
    t = _arr(t, np.float64)
    Phi = _arr(np.atleast_2d(Phi), np.float64)
    x = np.zeros(len(t))
    Mm = _arr(M, np.float64) if M is not None else None
    _check(lib().morap_project_down_hull(len(t), Phi.shape[0], _ptr(t, ctypes.c_double),
                                         _ptr(Phi, ctypes.c_double), _ptr(Mm, ctypes.c_double),
                                         _ptr(x, ctypes.c_double)))
    return x


def morap_task_preprocess(n_locs, q0, n_ap, delta, accepting):
    d = _arr(delta, np.int32)
    acc = _arr(accepting, np.uint8)
    n_out = ctypes.c_int32()
    flags = np.zeros(n_locs + 1, np.uint8)
    _check(lib().morap_task_preprocess(int(n_locs), int(q0), int(n_ap), _ptr(d, ctypes.c_int32),
                                       _ptr(acc, ctypes.c_uint8), ctypes.byref(n_out), _ptr(flags, ctypes.c_uint8)))
    return n_out.value, flags[: n_out.value]


def morap_product_info(ctx, p):
    info = np.zeros(10, np.int64)
    _check(lib().morap_product_info(ctx, int(p), _ptr(info, ctypes.c_int64)))
    keys = ["S", "Qn", "n_states", "n_sa", "n_trans", "init_local", "state_offset", "pre_begin", "agent", "task"]
    return dict(zip(keys, (int(v) for v in info)))


def morap_product_download(ctx, p):
    info = morap_product_info(ctx, p)
    ssa = np.zeros(info["n_states"] + 1, np.int64)
    satr = np.zeros(info["n_sa"] + 1, np.int64)
    col = np.zeros(max(info["n_trans"], 1), np.int32)
    prob = np.zeros(max(info["n_trans"], 1))
    cost = np.zeros(max(info["n_sa"], 1))
    loc = np.zeros(max(info["Qn"], 1), np.int32)
    _check(lib().morap_product_download(ctx, int(p), _ptr(ssa, ctypes.c_int64), _ptr(satr, ctypes.c_int64),
                                        _ptr(col, ctypes.c_int32), _ptr(prob, ctypes.c_double),
                                        _ptr(cost, ctypes.c_double), _ptr(loc, ctypes.c_int32)))
    return {"info": info, "state_sa": ssa, "sa_tr": satr, "col": col[: info["n_trans"]],
            "prob": prob[: info["n_trans"]], "cost": cost[: info["n_sa"]], "loc": loc[: info["Qn"]]}


def morap_product_locations(ctx, p):
    """The DFA location of each product location of product p (the state
    layout u = pl * S + s), without copying the CSR."""
    info = morap_product_info(ctx, p)
    loc = np.zeros(max(info["Qn"], 1), np.int32)
    _check(lib().morap_product_download(ctx, int(p), None, None, None, None, None, _ptr(loc, ctypes.c_int32)))
    return loc[: info["Qn"]]


def morap_last_policy(ctx, k, p):
    info = morap_product_info(ctx, p)
    mu = np.zeros(info["n_states"], np.uint8)
    v = np.zeros(info["n_states"])
    _check(lib().morap_last_policy(ctx, int(k), int(p), _ptr(mu, ctypes.c_uint8), _ptr(v, ctypes.c_double)))
    return mu, v


def morap_barrier_selfcheck(device=0):
    """Run the grid barrier's timeout self-check; returns (timed_out, ms)."""
    t = ctypes.c_int32()
    ms = ctypes.c_double()
    _check(lib().morap_barrier_selfcheck(int(device), ctypes.byref(t), ctypes.byref(ms)))
    return bool(t.value), ms.value


def morap_plain_vi_noalloc(n_states, n_sa, state_sa, sa_tr, col, prob, cost, pre_begin, init_state, w_cost, w_prob,
                           eps, tau, max_sweeps, values, policy, stream=None):
    """All array arguments are device addresses (ints); returns (code, c, sweeps)."""
    c = ctypes.c_double()
    sw = ctypes.c_int32()
    vp = lambda x: ctypes.c_void_p(int(x))
    code = lib().morap_plain_vi_noalloc(int(n_states), int(n_sa), vp(state_sa), vp(sa_tr), vp(col), vp(prob),
                                        vp(cost), int(pre_begin), int(init_state), float(w_cost), float(w_prob),
                                        float(eps), float(tau), int(max_sweeps), _stream(stream), vp(values),
                                        vp(policy), ctypes.byref(c), ctypes.byref(sw))
    if code not in (OK, ENOTCONV):
        _check(code)
    return code, c.value, sw.value


class Server:
    """Continuous-batching query server over built Contexts (morap_server_*)."""

    def __init__(self, contexts, max_batch=64, n_workers=8, eps=1e-6, max_iter=64, hbm_budget=0, merge_instances=0):
        cfg = ServerConfig()
        lib().morap_server_config_default(ctypes.byref(cfg))
        cfg.max_batch, cfg.n_workers, cfg.eps, cfg.max_iter, cfg.hbm_budget = max_batch, n_workers, eps, max_iter, \
            hbm_budget
        cfg.merge_instances = merge_instances
        self.contexts = list(contexts)
        self.n_obj = [c.n_agents + c.n_tasks for c in self.contexts]
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        self.h = ctypes.c_void_p()
        _check(lib().morap_server_create(arr, len(self.contexts), ctypes.byref(cfg), ctypes.byref(self.h)))
        self.max_iter = max_iter

    def submit(self, instance, t):
        t = _arr(t, np.float64)
        tk = ctypes.c_int64()
        _check(lib().morap_submit(self.h, int(instance), _ptr(t, ctypes.c_double), ctypes.byref(tk)))
        return tk.value

    def poll(self, ticket, instance):
        n = self.n_obj[instance]
        t_up, t_dn = np.zeros(n), np.zeros(n)
        res = PointResult()
        res.t_up = _ptr(t_up, ctypes.c_double)
        res.t_down = _ptr(t_dn, ctypes.c_double)
        code = lib().morap_poll(self.h, int(ticket), ctypes.byref(res))
        if code == EBUSY:
            return None
        _check(code)
        return {"feasible": bool(res.feasible), "iterations": res.iterations, "converged": bool(res.converged),
                "distance": res.distance, "t_up": t_up, "t_down": t_dn, "status": res.status}

    def wait(self, timeout_s=600.0):
        return lib().morap_server_wait(self.h, float(timeout_s))

    def stats(self):
        st = ServerStats()
        _check(lib().morap_server_stats(self.h, ctypes.byref(st)))
        return st.as_dict()

    def close(self):
        if self.h:
            lib().morap_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience


def add_agent_obj(ctx, a):
    """Add an object exposing the agent arrays (n_states, s0, state_ptr,
    sa_ptr, succ, prob, cost, label_ptr, label_ap)."""
    return morap_add_agent(ctx, a.n_states, a.s0, a.state_ptr, a.sa_ptr, a.succ, a.prob, a.cost, a.label_ptr,
                           a.label_ap)


def add_task_obj(ctx, t):
    return morap_add_task(ctx, t.n_locs, t.q0, t.n_ap, t.ap_ids, t.delta, t.accepting)


def torch_allocator_config(cfg, device=0):
    """Route the library's device allocations through PyTorch's caching
    allocator.  Keep the returned object alive as long as the context."""
    import torch

    def _alloc(nbytes, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device)
        except Exception:
            return None

    def _free(ptr, nbytes, user):
        torch.cuda.caching_allocator_delete(ptr)

    keep = (ALLOC_FN(_alloc), FREE_FN(_free))
    cfg.alloc, cfg.free = keep
    return keep


class Context:
    """Owns one morap_ctx (destroyed on close / garbage collection)."""

    def __init__(self, cfg=None, use_torch_allocator=False):
        self.cfg = cfg if cfg is not None else morap_config_default()
        self._keep = torch_allocator_config(self.cfg, self.cfg.device) if use_torch_allocator else None
        self.h = morap_ctx_create(self.cfg)
        self.n_agents = 0
        self.n_tasks = 0
        self.n_pairs = None  # set by select_pairs

    def add(self, agents, tasks):
        for a in agents:
            add_agent_obj(self.h, a)
            self.n_agents += 1
        for t in tasks:
            add_task_obj(self.h, t)
            self.n_tasks += 1
        return self

    def select_pairs(self, pairs):
        """Build only these (agent, task) products, in this order (before build)."""
        pairs = list(pairs)
        morap_select_pairs(self.h, [i for i, _ in pairs], [j for _, j in pairs])
        self.n_pairs = len(pairs)
        return self

    def build(self, stream=None):
        return morap_build(self.h, stream)

    def rebuild(self, stream=None):
        return morap_rebuild(self.h, stream)

    def solve(self, W, stream=None, evaluate=True, check=True):
        return morap_solve(self.h, W, self.n_agents, self.n_tasks, stream, evaluate, check, self.n_pairs)

    def supporting_points(self, W, stream=None, want_c=False, check=True):
        return morap_supporting_points(self.h, W, self.n_agents, self.n_tasks, stream, want_c, check)

    def query(self, t, M=None, eps=1e-6, max_iter=64, stream=None, check=True):
        """Algorithm 1 for threshold t; also returns the synthesis: `lambda`
        (convex weights of the points) and `assign_hist` (each point's task
        assignment); `random_assignment(...)` turns them into P[i][j]."""
        return morap_query(self.h, t, M, eps, max_iter, stream, check, n_tasks=self.n_tasks)

    def verify(self, t, M=None, eps=1e-6, max_iter=64, stream=None, check=True):
        """The verification-only loop (Sec. 5, Exp. 2): is t achievable?"""
        return morap_query(self.h, t, M, eps, max_iter, stream, check, n_tasks=self.n_tasks, verify_only=True)

    def stats(self):
        return morap_last_solve_stats(self.h)

    def close(self):
        if self.h:
            morap_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
