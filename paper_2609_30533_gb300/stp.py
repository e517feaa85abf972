"""ctypes binding of the C ABI in include/stp.h (argument marshalling only).

Every planning step runs in the CUDA library paper_2609_30533_gb300/_build/libstp.so;
importing a function here never falls back to Python or CPU code. If the library
is missing, ``lib()`` raises: build it with ``paper_2609_30533_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libstp.so")

STP_OK, STP_ERR_INVALID, STP_ERR_CAPACITY, STP_ERR_CUDA, STP_ERR_TIMEOUT, STP_NO_SOLUTION = range(6)
TRACE_INTS = 10
STP_LAUNCH_DEFAULT, STP_LAUNCH_STEPS, STP_LAUNCH_PERSISTENT = 0, 1, 2
STP_EDGES_DEVICE = 1
STP_EDGES_CLEARANCE = 2
STP_EDGES_NO_EARLY_EXIT = 4

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


class StpRobot(C.Structure):
    _fields_ = [("dof", C.c_int), ("arm", C.c_int), ("dh", _D), ("q_lo", _D), ("q_hi", _D),
                ("n_spheres", C.c_int), ("spheres", _D), ("v_max", C.c_double)]


class StpObstacles(C.Structure):
    _fields_ = [("n_obs", C.c_int), ("n_way", C.c_int), ("radius", _D), ("way", _D)]


class StpParams(C.Structure):
    _fields_ = [("variant", C.c_int), ("n_roots", C.c_int), ("ext_per_iter", C.c_int),
                ("max_iters", C.c_int), ("budget_ms", C.c_double), ("eta", C.c_double),
                ("edge_res", C.c_double), ("env_dt", C.c_double), ("p_new", C.c_double),
                ("p_guided", C.c_double), ("t_max", C.c_double), ("seed", C.c_ulonglong),
                ("problem_id", C.c_uint), ("precision", C.c_int), ("learned", C.c_int),
                ("capacity", C.c_int), ("iters_per_graph", C.c_int), ("t_offset", C.c_double),
                ("continuous", C.c_int), ("self_collision", C.c_int), ("launch_mode", C.c_int),
                ("persist_ctas", C.c_int)]


class StpStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("first_solution_iter", C.c_int), ("nodes", C.c_longlong),
                ("edges_validated", C.c_longlong), ("bridges_validated", C.c_longlong),
                ("root_checks", C.c_longlong), ("check_points", C.c_longlong), ("pair_tests", C.c_longlong),
                ("first_solution_ms", C.c_double), ("plan_ms", C.c_double), ("U", C.c_double),
                ("C", C.c_double), ("nn_evals", C.c_longlong), ("nn_nodes", C.c_longlong),
                ("bridge_evals", C.c_longlong), ("bridge_nodes", C.c_longlong), ("step_ms", C.c_double)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class StpBatchParams(C.Structure):
    _fields_ = [("nn_ctas", C.c_int), ("validate_ctas", C.c_int), ("iters_per_graph", C.c_int),
                ("launch_mode", C.c_int), ("team_ctas", C.c_int)]


class StpError(RuntimeError):
    def __init__(self, status, where, detail=""):
        self.status = status
        super().__init__("%s failed: %s%s" % (where, status_string(status), (" (" + detail + ")") if detail else ""))


_LIB = None


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("CUDA library not built: %s is missing (run paper_2609_30533_gb300.build.build())"
                           % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    L.stp_create_problem.argtypes = [C.POINTER(StpRobot), C.POINTER(StpObstacles), _D, _D, C.POINTER(StpParams),
                                     C.POINTER(C.c_void_p)]
    L.stp_create_problem.restype = C.c_int
    L.stp_plan.argtypes = [C.c_void_p, _D, _D, _I, _D, C.c_int, C.POINTER(StpStats)]
    L.stp_plan.restype = C.c_int
    L.stp_check_edges.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                  C.c_void_p, C.c_void_p, C.c_void_p]
    L.stp_check_edges.restype = C.c_int
    L.stp_free.argtypes = [C.c_void_p]
    L.stp_free.restype = None
    L.stp_release_cached.argtypes = []
    L.stp_release_cached.restype = None
    L.stp_set_stream.argtypes = [C.c_void_p, C.c_void_p]
    L.stp_set_stream.restype = C.c_int
    L.stp_status_string.argtypes = [C.c_int]
    L.stp_status_string.restype = C.c_char_p
    L.stp_last_error.argtypes = [C.c_void_p]
    L.stp_last_error.restype = C.c_char_p
    L.stp_last_validate.argtypes = [C.c_void_p, _D, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]
    L.stp_last_validate.restype = C.c_int
    L.stp_check_edges_noalloc.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
    L.stp_check_edges_noalloc.restype = C.c_int
    L.stp_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.POINTER(StpBatchParams), C.POINTER(C.c_void_p)]
    L.stp_batch_create.restype = C.c_int
    L.stp_batch_plan.argtypes = [C.c_void_p, C.POINTER(StpStats), _D]
    L.stp_batch_plan.restype = C.c_int
    L.stp_batch_path.argtypes = [C.c_void_p, C.c_int, _D, C.c_int, _I]
    L.stp_batch_path.restype = C.c_int
    L.stp_batch_free.argtypes = [C.c_void_p]
    L.stp_batch_free.restype = None
    L.stp_set_trace.argtypes = [C.c_void_p, C.c_int]
    L.stp_set_trace.restype = C.c_int
    L.stp_trace.argtypes = [C.c_void_p, _I, C.c_int, _I]
    L.stp_trace.restype = C.c_int
    L.stp_set_profiling.argtypes = [C.c_void_p, C.c_int]
    L.stp_set_profiling.restype = C.c_int
    L.stp_profile.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_char_p), _D, C.POINTER(C.c_longlong), _I]
    L.stp_profile.restype = C.c_int
    L.stp_tree_size.argtypes = [C.c_void_p, C.c_int, _I]
    L.stp_tree_size.restype = C.c_int
    L.stp_tree_nodes.argtypes = [C.c_void_p, C.c_int, _D, _I, _D, _D, _I, _I]
    L.stp_tree_nodes.restype = C.c_int
    L.stp_history.argtypes = [C.c_void_p, _D, C.c_int, _I]
    L.stp_history.restype = C.c_int
    L.stp_slots.argtypes = [C.c_void_p, _D, _I, _I, _I]
    L.stp_slots.restype = C.c_int
    L.stp_goal_grid.argtypes = [C.c_void_p, C.POINTER(C.c_long), _I, C.c_void_p, C.c_int]
    L.stp_goal_grid.restype = C.c_int
    _F = C.POINTER(C.c_float)
    L.stp_mlp_create.argtypes = [C.c_int, C.POINTER(C.c_void_p)]
    L.stp_mlp_create.restype = C.c_int
    L.stp_mlp_free.argtypes = [C.c_void_p]
    L.stp_mlp_free.restype = None
    L.stp_mlp_set_stream.argtypes = [C.c_void_p, C.c_void_p]
    L.stp_mlp_set_stream.restype = C.c_int
    L.stp_mlp_set_params.argtypes = [C.c_void_p, _F]
    L.stp_mlp_set_params.restype = C.c_int
    L.stp_mlp_get_params.argtypes = [C.c_void_p, _F]
    L.stp_mlp_get_params.restype = C.c_int
    L.stp_mlp_forward.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]
    L.stp_mlp_forward.restype = C.c_int
    L.stp_mlp_gradients.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, _F, _F, C.c_int]
    L.stp_mlp_gradients.restype = C.c_int
    L.stp_mlp_train_step.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_float, _F, C.c_int]
    L.stp_mlp_train_step.restype = C.c_int
    L.stp_mlp_set_profiling.argtypes = [C.c_void_p, C.c_int]
    L.stp_mlp_set_profiling.restype = C.c_int
    L.stp_mlp_profile.argtypes = [C.c_void_p, _D, _D, _D]
    L.stp_mlp_profile.restype = C.c_int
    L.stp_mlp_profile_step.argtypes = [C.c_void_p, _D, C.POINTER(C.c_int)]
    L.stp_mlp_profile_step.restype = C.c_int
    L.stp_mlp_last_error.argtypes = [C.c_void_p]
    L.stp_mlp_last_error.restype = C.c_char_p
    L.stp_problem_features.argtypes = [C.c_void_p, _F]
    L.stp_problem_features.restype = C.c_int
    L.stp_set_proposal.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    L.stp_set_proposal.restype = C.c_int
    L.stp_problem_targets.argtypes = [C.c_void_p, _F]
    L.stp_problem_targets.restype = C.c_int
    L.stp_selftest_bounded_wait.argtypes = [C.c_ulonglong, _I]
    L.stp_selftest_bounded_wait.restype = C.c_int
    _LIB = L
    return L


EXPORTED = ["stp_create_problem", "stp_plan", "stp_check_edges", "stp_free", "stp_set_stream",
            "stp_status_string", "stp_last_error", "stp_last_validate", "stp_set_profiling", "stp_profile",
            "stp_tree_size", "stp_tree_nodes", "stp_history", "stp_slots", "stp_goal_grid",
            "stp_check_edges_noalloc", "stp_batch_create", "stp_batch_plan", "stp_batch_path", "stp_batch_free",
            "stp_mlp_create", "stp_mlp_free", "stp_mlp_set_stream", "stp_mlp_set_params", "stp_mlp_get_params",
            "stp_mlp_forward", "stp_mlp_gradients", "stp_mlp_train_step", "stp_mlp_set_profiling",
            "stp_mlp_profile", "stp_mlp_profile_step", "stp_mlp_last_error", "stp_problem_features", "stp_set_proposal",
            "stp_problem_targets", "stp_selftest_bounded_wait", "stp_release_cached", "stp_set_trace", "stp_trace"]


def release_cached() -> None:
    """stp_release_cached: return the library's cached device blocks and streams."""
    lib().stp_release_cached()


def status_string(s: int) -> str:
    try:
        return lib().stp_status_string(int(s)).decode()
    except Exception:  # library missing: still name the code
        names = ["STP_OK", "STP_ERR_INVALID", "STP_ERR_CAPACITY", "STP_ERR_CUDA", "STP_ERR_TIMEOUT",
                 "STP_NO_SOLUTION"]
        return names[s] if 0 <= s < len(names) else str(s)


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


@dataclasses.dataclass
class PlanOutput:
    status: int
    U: float
    C: float
    path: np.ndarray
    stats: dict


class Problem:
    """Owns one stp_problem handle. Arrays are float64 numpy; see include/stp.h."""

    def __init__(self, *, dof, arm, dh, q_lo, q_hi, spheres, v_max, obs_radius, obs_way, q_start, q_goal,
                 variant=0, n_roots=4, ext_per_iter=64, max_iters=100, budget_ms=0.0, eta=0.1, edge_res=0.01,
                 env_dt=0.02, p_new=0.05, p_guided=0.95, t_max=10.0, seed=0, problem_id=0, precision=0,
                 capacity=0, iters_per_graph=0, learned=0, t_offset=0.0, continuous=0, self_collision=0,
                 launch_mode=0, persist_ctas=0):
        L = lib()
        self.dof = int(dof)
        self.precision = int(precision)
        self._keep = []

        def arr(x, shape=None):
            a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
            if shape is not None:
                a = a.reshape(shape)
            self._keep.append(a)
            return a

        dh_a = arr(dh if dh is not None else np.zeros((dof, 4)))
        robot = StpRobot(self.dof, 1 if arm else 0, _dp(dh_a) if arm else None, _dp(arr(q_lo)), _dp(arr(q_hi)),
                         len(spheres), _dp(arr(spheres)), float(v_max))
        obs_r = arr(obs_radius)
        way = arr(obs_way)
        obstacles = StpObstacles(len(obs_r), way.shape[1] if way.ndim == 3 else 1,
                                 _dp(obs_r) if len(obs_r) else None, _dp(way) if len(obs_r) else None)
        self.params = StpParams(int(variant), int(n_roots), int(ext_per_iter), int(max_iters), float(budget_ms),
                                float(eta), float(edge_res), float(env_dt), float(p_new), float(p_guided),
                                float(t_max), int(seed), int(problem_id), int(precision), int(learned),
                                int(capacity), int(iters_per_graph), float(t_offset), int(continuous),
                                int(self_collision), int(launch_mode), int(persist_ctas))
        h = C.c_void_p()
        s = L.stp_create_problem(C.byref(robot), C.byref(obstacles), _dp(arr(q_start)), _dp(arr(q_goal)),
                                 C.byref(self.params), C.byref(h))
        if s != STP_OK:
            raise StpError(s, "stp_create_problem", L.stp_last_error(None).decode())
        self.handle = h
        self.n_roots = int(n_roots)
        self.workers = int(ext_per_iter)

    def close(self):
        if getattr(self, "handle", None):
            lib().stp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return lib().stp_last_error(self.handle).decode()

    def set_stream(self, stream_ptr: Optional[int]):
        s = lib().stp_set_stream(self.handle, C.c_void_p(stream_ptr) if stream_ptr else None)
        if s != STP_OK:
            raise StpError(s, "stp_set_stream")

    def plan(self, cap: int = 1 << 16) -> PlanOutput:
        U = C.c_double()
        Cc = C.c_double()
        n = C.c_int()
        path = np.zeros((cap, self.dof + 1))
        st = StpStats()
        s = lib().stp_plan(self.handle, C.byref(U), C.byref(Cc), C.byref(n), _dp(path), cap, C.byref(st))
        if s not in (STP_OK, STP_NO_SOLUTION):
            raise StpError(s, "stp_plan", self.last_error())
        return PlanOutput(s, U.value, Cc.value, path[:n.value].copy(), st.as_dict())

    def check_edges(self, qa, ta, qb, tb, *, clearance=False, early_exit=True, n_checks=False):
        """Host arrays (numpy) of the precision type; returns verdict (uint8, 1 = free),
        clearance (or None) and check counts (or None)."""
        dt = np.float32 if self.precision == 0 else np.float64
        qa = np.ascontiguousarray(qa, dtype=dt)
        qb = np.ascontiguousarray(qb, dtype=dt)
        ta = np.ascontiguousarray(ta, dtype=dt)
        tb = np.ascontiguousarray(tb, dtype=dt)
        n = len(ta)
        ver = np.zeros(n, dtype=np.uint8)
        clr = np.zeros(n, dtype=dt) if clearance else None
        nc = np.zeros(n, dtype=np.int32) if n_checks else None
        flags = (STP_EDGES_CLEARANCE if clearance else 0) | (0 if early_exit else STP_EDGES_NO_EARLY_EXIT)
        s = lib().stp_check_edges(self.handle, n, qa.ctypes.data, ta.ctypes.data, qb.ctypes.data, tb.ctypes.data,
                                  flags, ver.ctypes.data, clr.ctypes.data if clearance else None,
                                  nc.ctypes.data if n_checks else None)
        if s != STP_OK:
            raise StpError(s, "stp_check_edges", self.last_error())
        return ver, clr, nc

    def check_edges_device(self, qa_ptr, ta_ptr, qb_ptr, tb_ptr, n, verdict_ptr, clearance_ptr=None,
                           early_exit=True):
        """Device pointers (e.g. torch tensors' data_ptr()); asynchronous on the problem's stream."""
        flags = STP_EDGES_DEVICE | (STP_EDGES_CLEARANCE if clearance_ptr else 0) | \
            (0 if early_exit else STP_EDGES_NO_EARLY_EXIT)
        s = lib().stp_check_edges(self.handle, int(n), C.c_void_p(qa_ptr), C.c_void_p(ta_ptr), C.c_void_p(qb_ptr),
                                  C.c_void_p(tb_ptr), flags, C.c_void_p(verdict_ptr),
                                  C.c_void_p(clearance_ptr) if clearance_ptr else None, None)
        if s != STP_OK:
            raise StpError(s, "stp_check_edges", self.last_error())

    def last_validate(self):
        """(ms, check points, pair tests) of the last collision-kernel launch."""
        ms = C.c_double()
        pts = C.c_longlong()
        prs = C.c_longlong()
        s = lib().stp_last_validate(self.handle, C.byref(ms), C.byref(pts), C.byref(prs))
        if s != STP_OK:
            raise StpError(s, "stp_last_validate")
        return ms.value, pts.value, prs.value

    def set_profiling(self, on: bool):
        s = lib().stp_set_profiling(self.handle, 1 if on else 0)
        if s != STP_OK:
            raise StpError(s, "stp_set_profiling")

    def profile(self):
        """{kernel name: (total ms, launches)} of the last profiled plan."""
        cap = 16
        names = (C.c_char_p * cap)()
        ms = np.zeros(cap)
        la = (C.c_longlong * cap)()
        n = C.c_int()
        s = lib().stp_profile(self.handle, cap, names, _dp(ms), la, C.byref(n))
        if s != STP_OK:
            raise StpError(s, "stp_profile")
        return {names[k].decode(): (float(ms[k]), int(la[k])) for k in range(n.value)}

    def set_trace(self, max_iters: int):
        """Record per-worker decision records of the next plans (0: off)."""
        s = lib().stp_set_trace(self.handle, int(max_iters))
        if s != STP_OK:
            raise StpError(s, "stp_set_trace", self.last_error())

    def trace(self) -> np.ndarray:
        """Decision records [iters][W][TRACE_INTS] (int32) of the last plan."""
        n = C.c_int()
        s = lib().stp_trace(self.handle, None, 0, C.byref(n))
        if s != STP_OK:
            raise StpError(s, "stp_trace", self.last_error())
        rec = np.zeros((n.value, self.workers, TRACE_INTS), dtype=np.int32)
        if n.value:
            s = lib().stp_trace(self.handle, rec.ctypes.data_as(_I), n.value, C.byref(n))
            if s != STP_OK:
                raise StpError(s, "stp_trace", self.last_error())
        return rec

    def features(self) -> np.ndarray:
        """Proposal-network input x[32] of this problem."""
        x = np.zeros(MLP_IN, dtype=np.float32)
        s = lib().stp_problem_features(self.handle, x.ctypes.data_as(C.POINTER(C.c_float)))
        if s != STP_OK:
            raise StpError(s, "stp_problem_features")
        return x

    def targets(self):
        """Training targets [130] of the last plan's path, or None without one."""
        t = np.zeros(MLP_NTGT, dtype=np.float32)
        s = lib().stp_problem_targets(self.handle, t.ctypes.data_as(C.POINTER(C.c_float)))
        if s == STP_NO_SOLUTION:
            return None
        if s != STP_OK:
            raise StpError(s, "stp_problem_targets", self.last_error())
        return t

    def set_proposal(self, y):
        """Learned-branch proposal from a network output y[160] (host array)."""
        y = np.ascontiguousarray(y, dtype=np.float32)
        assert y.size == MLP_OUT
        s = lib().stp_set_proposal(self.handle, y.ctypes.data, 0)
        if s != STP_OK:
            raise StpError(s, "stp_set_proposal", self.last_error())

    def set_proposal_device(self, y_ptr: int):
        s = lib().stp_set_proposal(self.handle, C.c_void_p(y_ptr), MLP_DEVICE)
        if s != STP_OK:
            raise StpError(s, "stp_set_proposal", self.last_error())

    def tree(self, arena: int):
        n = C.c_int()
        s = lib().stp_tree_size(self.handle, int(arena), C.byref(n))
        if s != STP_OK:
            raise StpError(s, "stp_tree_size")
        n = n.value
        d = self.dof
        x = np.zeros((n, d + 1))
        par = np.zeros(n, dtype=np.int32)
        tr = np.zeros(n)
        co = np.zeros(n)
        tree = np.zeros(n, dtype=np.int32)
        it = np.zeros(n, dtype=np.int32)
        if n:
            s = lib().stp_tree_nodes(self.handle, int(arena), _dp(x), par.ctypes.data_as(_I), _dp(tr), _dp(co),
                                     tree.ctypes.data_as(_I), it.ctypes.data_as(_I))
            if s != STP_OK:
                raise StpError(s, "stp_tree_nodes")
        return dict(x=x, parent=par, troot=tr, cost=co, tree=tree, iter=it)

    def history(self):
        n = C.c_int()
        lib().stp_history(self.handle, None, 0, C.byref(n))
        U = np.zeros(max(n.value, 1))
        lib().stp_history(self.handle, _dp(U), n.value, C.byref(n))
        return U[:n.value]

    def slots(self):
        N = self.n_roots
        T = np.zeros(N)
        hr = np.zeros(N, dtype=np.int32)
        ac = np.zeros(N, dtype=np.int32)
        gen = np.zeros(N, dtype=np.int32)
        s = lib().stp_slots(self.handle, _dp(T), hr.ctypes.data_as(_I), ac.ctypes.data_as(_I),
                            gen.ctypes.data_as(_I))
        if s != STP_OK:
            raise StpError(s, "stp_slots")
        return dict(T=T, has_root=hr, active=ac, gen=gen)

    def goal_grid(self):
        kmin = C.c_long()
        n = C.c_int()
        lib().stp_goal_grid(self.handle, C.byref(kmin), C.byref(n), None, 0)
        f = np.zeros(max(n.value, 1), dtype=np.uint8)
        lib().stp_goal_grid(self.handle, C.byref(kmin), C.byref(n), f.ctypes.data, n.value)
        return kmin.value, f[:n.value]


def problem_from(prob, params, **over) -> Problem:
    """Build a Problem from objects with the fields of workloads.Problem / Params."""
    kw = dict(variant=params.variant, n_roots=params.n_roots, ext_per_iter=params.workers,
              max_iters=params.max_iters, eta=params.eta, edge_res=params.res, env_dt=params.dt,
              p_new=params.p_new, p_guided=params.p_guided, t_max=params.H, seed=params.seed,
              problem_id=params.problem_id, self_collision=1 if getattr(prob, "self_collision", False) else 0)
    kw.update(over)
    return Problem(dof=prob.dof, arm=prob.arm, dh=prob.dh, q_lo=prob.qlo, q_hi=prob.qhi, spheres=prob.spheres,
                   v_max=prob.vmax, obs_radius=prob.obs_r, obs_way=prob.way, q_start=prob.qs, q_goal=prob.qg,
                   **kw)


class Batch:
    """Many FP32 problems planned together (stp_batch_*). The problems must stay
    alive while the batch exists."""

    def __init__(self, problems, nn_ctas=0, validate_ctas=0, iters_per_graph=0, launch_mode=0, team_ctas=0):
        L = lib()
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p.handle.value for p in self.problems])
        bp = StpBatchParams(int(nn_ctas), int(validate_ctas), int(iters_per_graph), int(launch_mode),
                            int(team_ctas))
        h = C.c_void_p()
        s = L.stp_batch_create(arr, len(self.problems), C.byref(bp), C.byref(h))
        if s != STP_OK:
            raise StpError(s, "stp_batch_create", L.stp_last_error(None).decode())
        self.handle = h

    def plan(self):
        """Returns (batch_ms, [stats dict per problem])."""
        n = len(self.problems)
        st = (StpStats * n)()
        ms = C.c_double()
        s = lib().stp_batch_plan(self.handle, st, C.byref(ms))
        if s != STP_OK:
            raise StpError(s, "stp_batch_plan", lib().stp_last_error(None).decode())
        return ms.value, [st[i].as_dict() for i in range(n)]

    def path(self, i, cap=1 << 16):
        dof = self.problems[i].dof
        buf = np.zeros((cap, dof + 1))
        n = C.c_int()
        s = lib().stp_batch_path(self.handle, int(i), _dp(buf), cap, C.byref(n))
        if s != STP_OK:
            raise StpError(s, "stp_batch_path")
        return buf[:n.value].copy()

    def close(self):
        if getattr(self, "handle", None):
            lib().stp_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Learned proposal network (stp_mlp_*).
# ---------------------------------------------------------------------------
MLP_IN, MLP_OUT, MLP_NTGT, MLP_NPARAM = 32, 160, 130, 181152
MLP_DEVICE = 1
_MLP_SHAPES = (("W1", (256, 32)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)),
               ("b3", (256,)), ("W4", (160, 256)), ("b4", (160,)))


def flatten_params(P) -> np.ndarray:
    """dict of arrays (oracle layout) -> STP_MLP_NPARAM float32 vector."""
    return np.concatenate([np.asarray(P[k], dtype=np.float32)[:s[0]].reshape(-1) if k in ("W4", "b4")
                           else np.asarray(P[k], dtype=np.float32).reshape(-1) for k, s in _MLP_SHAPES])


def unflatten_params(v) -> dict:
    out, o = {}, 0
    for k, s in _MLP_SHAPES:
        n = int(np.prod(s))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(s)
        o += n
    return out


class Mlp:
    """The proposal network on the device (stp_mlp_*)."""

    def __init__(self, max_batch: int):
        L = lib()
        h = C.c_void_p()
        s = L.stp_mlp_create(int(max_batch), C.byref(h))
        if s != STP_OK:
            raise StpError(s, "stp_mlp_create", L.stp_mlp_last_error(None).decode())
        self.handle = h
        self.max_batch = int(max_batch)

    def _err(self, s, where):
        return StpError(s, where, lib().stp_mlp_last_error(self.handle).decode())

    def set_stream(self, stream_ptr):
        lib().stp_mlp_set_stream(self.handle, C.c_void_p(stream_ptr) if stream_ptr else None)

    def set_params(self, flat: np.ndarray):
        v = np.ascontiguousarray(flat, dtype=np.float32)
        assert v.size == MLP_NPARAM
        s = lib().stp_mlp_set_params(self.handle, v.ctypes.data_as(C.POINTER(C.c_float)))
        if s != STP_OK:
            raise self._err(s, "stp_mlp_set_params")

    def get_params(self) -> np.ndarray:
        v = np.zeros(MLP_NPARAM, dtype=np.float32)
        s = lib().stp_mlp_get_params(self.handle, v.ctypes.data_as(C.POINTER(C.c_float)))
        if s != STP_OK:
            raise self._err(s, "stp_mlp_get_params")
        return v

    def forward(self, X: np.ndarray) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        B = X.shape[0]
        Y = np.zeros((B, MLP_OUT), dtype=np.float32)
        s = lib().stp_mlp_forward(self.handle, B, X.ctypes.data, Y.ctypes.data, 0)
        if s != STP_OK:
            raise self._err(s, "stp_mlp_forward")
        return Y

    def forward_device(self, B: int, x_ptr: int, y_ptr: int):
        s = lib().stp_mlp_forward(self.handle, int(B), C.c_void_p(x_ptr), C.c_void_p(y_ptr), MLP_DEVICE)
        if s != STP_OK:
            raise self._err(s, "stp_mlp_forward")

    def gradients(self, X: np.ndarray, T: np.ndarray):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        g = np.zeros(MLP_NPARAM, dtype=np.float32)
        loss = C.c_float()
        s = lib().stp_mlp_gradients(self.handle, X.shape[0], X.ctypes.data, T.ctypes.data, C.byref(loss),
                                    g.ctypes.data_as(C.POINTER(C.c_float)), 0)
        if s != STP_OK:
            raise self._err(s, "stp_mlp_gradients")
        return float(loss.value), g

    def train_step(self, X: np.ndarray, T: np.ndarray, lr: float) -> float:
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        loss = C.c_float()
        s = lib().stp_mlp_train_step(self.handle, X.shape[0], X.ctypes.data, T.ctypes.data, float(lr),
                                     C.byref(loss), 0)
        if s != STP_OK:
            raise self._err(s, "stp_mlp_train_step")
        return float(loss.value)

    def train_step_device(self, B: int, x_ptr: int, t_ptr: int, lr: float) -> float:
        loss = C.c_float()
        s = lib().stp_mlp_train_step(self.handle, int(B), C.c_void_p(x_ptr), C.c_void_p(t_ptr), float(lr),
                                     C.byref(loss), MLP_DEVICE)
        if s != STP_OK:
            raise self._err(s, "stp_mlp_train_step")
        return float(loss.value)

    def set_profiling(self, on: bool):
        lib().stp_mlp_set_profiling(self.handle, 1 if on else 0)

    def profile(self):
        """(GEMM ms, FLOPs, algorithmic bytes) since the last call."""
        ms, fl, by = C.c_double(), C.c_double(), C.c_double()
        lib().stp_mlp_profile(self.handle, C.byref(ms), C.byref(fl), C.byref(by))
        return ms.value, fl.value, by.value

    def profile_step(self):
        """(device ms of whole training steps, steps) since the last call."""
        ms, n = C.c_double(), C.c_int()
        s = lib().stp_mlp_profile_step(self.handle, C.byref(ms), C.byref(n))
        if s != STP_OK:
            raise StpError(s, "stp_mlp_profile_step")
        return ms.value, n.value

    def close(self):
        if getattr(self, "handle", None):
            lib().stp_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_bounded_wait(limit_ns: int):
    """(status, microseconds waited) of the bounded-wait self-test."""
    us = C.c_int()
    s = lib().stp_selftest_bounded_wait(C.c_ulonglong(limit_ns), C.byref(us))
    return s, us.value
