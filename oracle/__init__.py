"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this package. The planner library never imports or links it.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import functools
from typing import Dict, List

import numpy as np

from . import build as _build

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_U8 = C.POINTER(C.c_ubyte)


class OrcProblem(C.Structure):
    _fields_ = [("dof", C.c_int), ("arm", C.c_int), ("dh", _D), ("qlo", _D), ("qhi", _D),
                ("n_sph", C.c_int), ("sph", _D), ("vmax", C.c_double), ("n_obs", C.c_int),
                ("n_way", C.c_int), ("obs_r", _D), ("way", _D), ("qs", _D), ("qg", _D),
                ("self_collision", C.c_int)]


class OrcParams(C.Structure):
    _fields_ = [("variant", C.c_int), ("n_roots", C.c_int), ("workers", C.c_int),
                ("max_iters", C.c_int), ("eta", C.c_double), ("res", C.c_double),
                ("dt", C.c_double), ("p_new", C.c_double), ("p_guided", C.c_double),
                ("H", C.c_double), ("seed", C.c_ulonglong), ("problem_id", C.c_uint),
                ("flag_tol", C.c_double), ("flag_clear", C.c_double), ("learned", C.c_int),
                ("proposal", _D), ("t_offset", C.c_double), ("continuous", C.c_int),
                ("follow_rec", _I), ("follow_iters", C.c_int), ("follow_grid", _U8), ("follow_nk", C.c_int)]


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


@functools.lru_cache(maxsize=1)
def lib():
    path = _build.build()
    L = C.CDLL(path)
    L.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint), C.POINTER(C.c_uint), C.POINTER(C.c_uint)]
    L.orc_fk.argtypes = [C.POINTER(OrcProblem), _D, _D, _D, _D]
    L.orc_obstacle_position.argtypes = [C.POINTER(OrcProblem), C.c_int, C.c_double, _D]
    L.orc_state_free.argtypes = [C.POINTER(OrcProblem), _D, C.c_double, _D]
    L.orc_state_free.restype = C.c_int
    L.orc_check_edges.argtypes = [C.POINTER(OrcProblem), C.c_int, _D, _D, _D, _D, C.c_double, _U8,
                                  _D, _I, _D, _D]
    L.orc_interval_partition.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                                         C.c_long, C.c_int, _U8, _D, _D, _D, C.c_int]
    L.orc_interval_partition.restype = C.c_int
    L.orc_interval_sample.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int, C.c_double,
                                      C.c_long, C.c_int, _U8, C.c_int, C.c_double, C.c_double,
                                      C.c_double, _I]
    L.orc_interval_sample.restype = C.c_double
    L.orc_recycle_update.argtypes = [C.c_int, _D, _I, _I, _I, C.c_double, C.c_long, C.c_int, _U8,
                                     C.c_double]
    L.orc_recycle_update.restype = C.c_int
    L.orc_plan.argtypes = [C.POINTER(OrcProblem), C.POINTER(OrcParams), C.POINTER(C.c_void_p)]
    L.orc_learned_sample.argtypes = [_D, _D, _D, _D, _D, C.c_int, C.c_double, C.c_ulonglong, C.c_uint, C.c_uint,
                                     C.c_uint, _I, _D, _D]
    L.orc_learned_sample.restype = C.c_int
    L.orc_self_pairs.argtypes = [C.POINTER(OrcProblem), _I, C.c_int]
    L.orc_self_pairs.restype = C.c_int
    L.orc_check_edges_continuous.argtypes = [C.POINTER(OrcProblem), C.c_int, _D, _D, _D, _D, _U8, _D]
    L.orc_check_edges_continuous.restype = C.c_int
    L.orc_plan.restype = C.c_int
    L.orc_result_summary.argtypes = [C.c_void_p, _D]
    L.orc_result_path.argtypes = [C.c_void_p, _D]
    L.orc_result_arena_size.argtypes = [C.c_void_p, C.c_int]
    L.orc_result_arena_size.restype = C.c_int
    L.orc_result_arena.argtypes = [C.c_void_p, C.c_int, _D, _I, _D, _D, _I, _I]
    L.orc_result_history.argtypes = [C.c_void_p, _D, _D, _D]
    L.orc_nn_spacetime.argtypes = [C.c_int, C.c_int, _D, _D, C.c_int, C.c_double, _D, C.c_double,
                                   C.c_int, C.c_double, _D]
    L.orc_nn_spacetime.restype = C.c_int
    L.orc_result_margin_types.argtypes = [C.c_void_p, _D]
    L.orc_result_slots.argtypes = [C.c_void_p, _D, _I, _I, _I]
    L.orc_result_trees.argtypes = [C.c_void_p, _I, _D]
    L.orc_result_goal_grid.argtypes = [C.c_void_p, C.POINTER(C.c_long), _D, C.c_int]
    L.orc_result_goal_grid.restype = C.c_int
    L.orc_result_incumbent.argtypes = [C.c_void_p, _I, _I, _I]
    L.orc_result_C_history.argtypes = [C.c_void_p, _D]
    L.orc_result_trace.argtypes = [C.c_void_p, _I, _D]
    L.orc_result_follow.argtypes = [C.c_void_p, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), _I, C.c_int]
    L.orc_result_follow.restype = C.c_int
    L.orc_follow_kinds.argtypes = []
    L.orc_follow_kinds.restype = C.c_int
    L.orc_nn_config.argtypes = [C.c_int, C.c_int, _D, _D, _D]
    L.orc_nn_config.restype = C.c_int
    L.orc_publish_winner.argtypes = [C.c_int, _D, _D, _I]
    L.orc_publish_winner.restype = C.c_int
    L.orc_bridge.argtypes = [C.POINTER(OrcProblem), _D, C.c_double, C.c_double, C.c_double, C.c_int, C.c_int, _D,
                             _D, _D, _I, C.c_double, C.c_double, C.c_double, _I, _D]
    L.orc_bridge.restype = C.c_int
    L.orc_result_free.argtypes = [C.c_void_p]
    return L


# Decision records (one per worker and iteration), the layout shared with the
# device library's trace: see TRACE_FIELDS / TRACE_FLAGS.
TRACE_INTS = 10
TRACE_FIELDS = ("flags", "group", "parent", "ext_count", "br_set", "br_idx", "br_count", "inserted",
                "component", "T_bits")
TRACE_FLAGS = {"fwd": 1, "sampled": 2, "virtual": 4, "emit": 8, "root_hit": 16, "ext_hit": 32,
               "inserted": 64, "br_cand": 128, "br_emit": 256, "br_hit": 512, "winner": 1024,
               "learned": 2048, "learned_T": 4096, "guided": 8192}
FOLLOW_KINDS = ("direction", "group", "learned_component", "learned_T", "root", "window", "virtual",
                "parent", "emit", "ext_count", "ext_hit", "inserted", "br_cand", "br_emit", "br_count",
                "br_hit", "winner", "grid", "guided", "goal_time")


class _ProblemHandle:
    """Keeps the numpy buffers alive for an OrcProblem struct."""

    def __init__(self, prob):
        self.bufs = []

        def keep(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            self.bufs.append(a)
            return _dptr(a)

        dh = prob.dh if prob.dh is not None else np.zeros((prob.dof, 4))
        self.s = OrcProblem(prob.dof, 1 if prob.arm else 0, keep(dh), keep(prob.qlo), keep(prob.qhi),
                            len(prob.spheres), keep(prob.spheres), float(prob.vmax),
                            len(prob.obs_r), prob.way.shape[1], keep(prob.obs_r), keep(prob.way),
                            keep(prob.qs), keep(prob.qg), 1 if getattr(prob, "self_collision", False) else 0)

    @property
    def ref(self):
        return C.byref(self.s)


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def fk(prob, q):
    h = _ProblemHandle(prob)
    S = len(prob.spheres)
    nf = prob.dof + 1 if prob.arm else 1
    cen = np.zeros((S, 3))
    org = np.zeros((nf, 3))
    rot = np.zeros((nf, 9))
    q = np.ascontiguousarray(q, dtype=np.float64)
    lib().orc_fk(h.ref, _dptr(q), _dptr(cen), _dptr(org), _dptr(rot))
    return cen, org, rot.reshape(nf, 3, 3)


def obstacle_position(prob, m, t):
    h = _ProblemHandle(prob)
    o = np.zeros(3)
    lib().orc_obstacle_position(h.ref, int(m), float(t), _dptr(o))
    return o


def state_free(prob, q, t):
    h = _ProblemHandle(prob)
    q = np.ascontiguousarray(q, dtype=np.float64)
    clr = C.c_double()
    ok = lib().orc_state_free(h.ref, _dptr(q), float(t), C.byref(clr))
    return bool(ok), clr.value


def check_edges(prob, qa, ta, qb, tb, res, bounds=False):
    """FP64 verdicts (1 = free), clearance, check-point count and the distance
    of the check-count argument from an integer, for a batch of edges; with
    bounds=True also the signed margin of the checked states from the
    configuration-box boundary."""
    h = _ProblemHandle(prob)
    qa = np.ascontiguousarray(qa, dtype=np.float64)
    qb = np.ascontiguousarray(qb, dtype=np.float64)
    ta = np.ascontiguousarray(ta, dtype=np.float64)
    tb = np.ascontiguousarray(tb, dtype=np.float64)
    n = len(ta)
    v = np.zeros(n, dtype=np.uint8)
    clr = np.zeros(n)
    nc = np.zeros(n, dtype=np.int32)
    im = np.zeros(n)
    bm = np.zeros(n)
    lib().orc_check_edges(h.ref, n, _dptr(qa), _dptr(ta), _dptr(qb), _dptr(tb), float(res),
                          v.ctypes.data_as(_U8), _dptr(clr), nc.ctypes.data_as(_I), _dptr(im), _dptr(bm))
    if bounds:
        return v, clr, nc, im, bm
    return v, clr, nc, im


def nn_spacetime(x, qr, tr, sigma, vmax, troot=None, U=float("inf")):
    """Index of argmin rho_sigma over nodes x [n][d+1] (or -1) and the value."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, d1 = x.shape
    qr = np.ascontiguousarray(qr, dtype=np.float64)
    tro = np.ascontiguousarray(troot if troot is not None else np.zeros(n), dtype=np.float64)
    rho = C.c_double()
    i = lib().orc_nn_spacetime(n, d1 - 1, _dptr(x), _dptr(tro), 1 if troot is not None else 0, float(U),
                               _dptr(qr), float(tr), int(sigma), float(vmax), C.byref(rho))
    return i, rho.value


def interval_partition(Lg, H, dt, N, U, kmin, free_flags):
    f = np.ascontiguousarray(free_flags, dtype=np.uint8)
    uni = np.zeros(N)
    w = C.c_double()
    cap = len(f) + N + 4
    pcs = np.zeros((cap, 3))
    n = lib().orc_interval_partition(float(Lg), float(H), float(dt), int(N), float(U), int(kmin), len(f),
                                     f.ctypes.data_as(_U8), _dptr(uni), C.byref(w), _dptr(pcs), cap)
    return uni, w.value, pcs[:n]


def interval_sample(Lg, H, dt, N, U, kmin, free_flags, group, u_coin, u_pos, p_guided):
    f = np.ascontiguousarray(free_flags, dtype=np.uint8)
    g = C.c_int()
    T = lib().orc_interval_sample(float(Lg), float(H), float(dt), int(N), float(U), int(kmin), len(f),
                                  f.ctypes.data_as(_U8), int(group), float(u_coin), float(u_pos),
                                  float(p_guided), C.byref(g))
    return T, bool(g.value)


def recycle_update(T, has_root, active, gen, U, kmin, free_flags, dt):
    T = np.array(T, dtype=np.float64)
    hr = np.array(has_root, dtype=np.int32)
    ac = np.array(active, dtype=np.int32)
    gn = np.array(gen, dtype=np.int32)
    f = np.ascontiguousarray(free_flags, dtype=np.uint8)
    n = lib().orc_recycle_update(len(T), _dptr(T), hr.ctypes.data_as(_I), ac.ctypes.data_as(_I),
                                 gn.ctypes.data_as(_I), float(U), int(kmin), len(f),
                                 f.ctypes.data_as(_U8), float(dt))
    return T, hr, ac, gn, n


@dataclasses.dataclass
class Arena:
    x: np.ndarray       # [n][dof+1]  (q..., t)
    parent: np.ndarray  # [n]
    troot: np.ndarray
    cost: np.ndarray
    tree: np.ndarray
    iter: np.ndarray


@dataclasses.dataclass
class PlanResult:
    U: float
    C: float
    iters: int
    first_iter: int
    ext_checked: int
    bridge_checked: int
    root_checked: int
    inserted: int
    path: np.ndarray
    status: int
    fwd: Arena
    seg: List[Arena]
    U_hist: np.ndarray
    margin_hist: np.ndarray
    clear_hist: np.ndarray
    margin_types: np.ndarray  # [iters][6] nn, count, interval, bounds, rank, clearance
    slots: Dict[str, np.ndarray]
    trees: Dict[str, np.ndarray]
    incumbent: tuple
    goal_kmin: int
    goal_clearance: np.ndarray
    C_hist: np.ndarray = None
    trace: np.ndarray = None     # [iters][W][TRACE_INTS] int32 decision records
    trace_d: np.ndarray = None   # [iters][W][4] (T, t_r, window lo, window hi), NaN where not drawn
    follow: Dict[str, object] = None  # follow mode: adopted / differing counts per kind, unflagged list


def make_params(params, proposal=None, t_offset=0.0, continuous=False, **over) -> OrcParams:
    p = dataclasses.replace(params, **over) if over else params
    prm = OrcParams(p.variant, p.n_roots, p.workers, p.max_iters, p.eta, p.res, p.dt, p.p_new,
                    p.p_guided, p.H, p.seed, p.problem_id, 0.0, 0.0, 0, None, float(t_offset),
                    1 if continuous else 0, None, 0, None, 0)
    if proposal is not None:
        prm.learned = 1
        prm.proposal = _dptr(proposal)
    return prm


def learned_sample(y, qlo, qhi, H, seed, problem_id, k, w, qs=None, qg=None):
    """Learned-branch draws of worker w at iteration k: (learned, waypoint
    index, q_r, T_l or NaN). Waypoint offsets are taken from the straight line
    between qs and qg (default: both at the box centre)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    lo = np.ascontiguousarray(qlo, dtype=np.float64)
    hi = np.ascontiguousarray(qhi, dtype=np.float64)
    d = len(lo)
    c = 0.5 * (lo + hi)
    s0 = np.ascontiguousarray(c if qs is None else qs, dtype=np.float64)
    g0 = np.ascontiguousarray(c if qg is None else qg, dtype=np.float64)
    qr = np.zeros(d)
    wi = C.c_int()
    Tl = C.c_double()
    f = lib().orc_learned_sample(_dptr(y), _dptr(lo), _dptr(hi), _dptr(s0), _dptr(g0), d, float(H),
                                 C.c_ulonglong(seed),
                                 C.c_uint(problem_id), C.c_uint(k), C.c_uint(w), C.byref(wi), _dptr(qr),
                                 C.byref(Tl))
    return bool(f), wi.value, qr, Tl.value


def plan(prob, params, proposal=None, t_offset=0.0, continuous=False, follow=None, **over) -> PlanResult:
    """proposal: network output y[160] (float64 array) enables the learned
    branch; t_offset: absolute time of the query's local time 0; continuous:
    closed-form edge validation (point robots); follow: (records
    [iters][W][TRACE_INTS] int32, goal-grid free flags or None) of a device run:
    the oracle adopts the device's choice at every flagged decision and records
    every unflagged difference (follow mode)."""
    L = lib()
    h = _ProblemHandle(prob)
    if proposal is not None:
        proposal = np.ascontiguousarray(proposal, dtype=np.float64)
    prm = make_params(params, proposal, t_offset, continuous, **over)
    keep = []
    if follow is not None:
        rec, grid = follow
        rec = np.ascontiguousarray(rec, dtype=np.int32)
        assert rec.ndim == 3 and rec.shape[1] == prm.workers and rec.shape[2] == TRACE_INTS, rec.shape
        keep.append(rec)
        prm.follow_rec = rec.ctypes.data_as(_I)
        prm.follow_iters = rec.shape[0]
        if grid is not None:
            grid = np.ascontiguousarray(grid, dtype=np.uint8)
            keep.append(grid)
            prm.follow_grid = grid.ctypes.data_as(_U8)
            prm.follow_nk = len(grid)
    handle = C.c_void_p()
    L.orc_plan(h.ref, C.byref(prm), C.byref(handle))
    try:
        s = np.zeros(12)
        L.orc_result_summary(handle, _dptr(s))
        d = prob.dof
        plen = int(s[8])
        path = np.zeros((plen, d + 1))
        if plen:
            L.orc_result_path(handle, _dptr(path))

        def arena(i):
            n = L.orc_result_arena_size(handle, i)
            x = np.zeros((n, d + 1))
            par = np.zeros(n, dtype=np.int32)
            tr = np.zeros(n)
            co = np.zeros(n)
            tree = np.zeros(n, dtype=np.int32)
            it = np.zeros(n, dtype=np.int32)
            if n:
                L.orc_result_arena(handle, i, _dptr(x), par.ctypes.data_as(_I), _dptr(tr), _dptr(co),
                                   tree.ctypes.data_as(_I), it.ctypes.data_as(_I))
            return Arena(x, par, tr, co, tree, it)

        iters = int(s[2])
        Uh = np.zeros(iters)
        Mh = np.zeros(iters)
        Ch = np.zeros(iters)
        MT = np.zeros((iters, 6))
        if iters:
            L.orc_result_history(handle, _dptr(Uh), _dptr(Mh), _dptr(Ch))
            L.orc_result_margin_types(handle, _dptr(MT))
        N = prm.n_roots
        sl = {"T": np.zeros(N), "has_root": np.zeros(N, dtype=np.int32),
              "active": np.zeros(N, dtype=np.int32), "gen": np.zeros(N, dtype=np.int32)}
        if prm.variant != 0:
            L.orc_result_slots(handle, _dptr(sl["T"]), sl["has_root"].ctypes.data_as(_I),
                               sl["active"].ctypes.data_as(_I), sl["gen"].ctypes.data_as(_I))
        nt = int(s[10])
        tr = {"group": np.zeros(nt, dtype=np.int32), "T": np.zeros(nt)}
        if nt:
            L.orc_result_trees(handle, tr["group"].ctypes.data_as(_I), _dptr(tr["T"]))
        f, sg, b = C.c_int(), C.c_int(), C.c_int()
        L.orc_result_incumbent(handle, C.byref(f), C.byref(sg), C.byref(b))
        kmin = C.c_long()
        gcap = 1 << 20
        gcl = np.zeros(gcap)
        ng = L.orc_result_goal_grid(handle, C.byref(kmin), _dptr(gcl), gcap)
        Chh = np.zeros(iters)
        W = prm.workers
        trace = np.zeros((iters, W, TRACE_INTS), dtype=np.int32)
        trace_d = np.zeros((iters, W, 4))
        if iters:
            L.orc_result_C_history(handle, _dptr(Chh))
            L.orc_result_trace(handle, trace.ctypes.data_as(_I), _dptr(trace_d))
        nk = L.orc_follow_kinds()
        fo = np.zeros(nk, dtype=np.int64)
        fd = np.zeros(nk, dtype=np.int64)
        nu = L.orc_result_follow(handle, fo.ctypes.data_as(C.POINTER(C.c_longlong)),
                                 fd.ctypes.data_as(C.POINTER(C.c_longlong)), None, 0)
        un = np.zeros((max(nu, 1), 3), dtype=np.int32)
        L.orc_result_follow(handle, None, None, un.ctypes.data_as(_I), nu)
        follow_info = None
        if follow is not None:
            follow_info = {"followed": dict(zip(FOLLOW_KINDS, fo.tolist())),
                           "flagged_diff": dict(zip(FOLLOW_KINDS, fd.tolist())),
                           "unflagged": [(int(a), int(b), FOLLOW_KINDS[c]) for a, b, c in un[:nu]]}
        return PlanResult(U=s[0], C=s[1], iters=iters, first_iter=int(s[3]), ext_checked=int(s[4]),
                          bridge_checked=int(s[5]), root_checked=int(s[6]), inserted=int(s[7]),
                          path=path, status=int(s[11]), fwd=arena(-1),
                          seg=[arena(i) for i in range(N)], U_hist=Uh, margin_hist=Mh, clear_hist=Ch,
                          margin_types=MT, slots=sl, trees=tr, incumbent=(f.value, sg.value, b.value),
                          goal_kmin=kmin.value, goal_clearance=gcl[:ng].copy(), C_hist=Chh, trace=trace,
                          trace_d=trace_d, follow=follow_info)
    finally:
        L.orc_result_free(handle)


def plan_sequence(prob, params, goals, **over):
    """Goal sequence as successive single-goal queries (Sec. "Problem
    Formulation"): query i starts at the previous arrival state with local time
    0, obstacle trajectories shifted by its absolute start time, and the
    remaining horizon. Returns (status, path [n][d+1] in absolute time, visit
    times, per-query results)."""
    t_abs = 0.0
    q = np.asarray(prob.qs, float)
    segs, visits, results = [], [], []
    for i, g in enumerate(goals):
        H = params.H - t_abs
        if not H > 0:
            return 5, None, visits, results
        pi = dataclasses.replace(prob, qs=q.copy(), qg=np.asarray(g, float).copy())
        r = plan(pi, dataclasses.replace(params, H=H, problem_id=params.problem_id + i, **over), t_offset=t_abs)
        results.append(r)
        if r.status != 0:
            return r.status, None, visits, results
        path = r.path.copy()
        path[:, prob.dof] += t_abs
        segs.append(path if i == 0 else path[1:])
        t_abs += r.U
        visits.append(t_abs)
        q = np.asarray(g, float)
    return 0, np.concatenate(segs), visits, results


def check_edges_continuous(prob, qa, ta, qb, tb):
    """Closed-form verdicts (1 = free) and exact clearances of point-robot edges."""
    h = _ProblemHandle(prob)
    qa = np.ascontiguousarray(qa, dtype=np.float64)
    qb = np.ascontiguousarray(qb, dtype=np.float64)
    ta = np.ascontiguousarray(ta, dtype=np.float64)
    tb = np.ascontiguousarray(tb, dtype=np.float64)
    n = len(ta)
    v = np.zeros(n, dtype=np.uint8)
    clr = np.zeros(n)
    r = lib().orc_check_edges_continuous(h.ref, n, _dptr(qa), _dptr(ta), _dptr(qb), _dptr(tb),
                                         v.ctypes.data_as(_U8), _dptr(clr))
    if r != 0:
        raise ValueError("continuous validation needs a point robot")
    return v, clr


def self_pairs(prob) -> np.ndarray:
    """Self-collision sphere pairs [n][2] of an arm with self_collision set."""
    h = _ProblemHandle(prob)
    n = lib().orc_self_pairs(h.ref, None, 0)
    out = np.zeros((max(n, 1), 2), dtype=np.int32)
    lib().orc_self_pairs(h.ref, out.ctypes.data_as(_I), n)
    return out[:n]


def nn_config(x, qr):
    """Configuration-distance NN (root recycling) over configurations x [n][d]:
    (index or -1, distance); tie: lowest index."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, d = x.shape
    qr = np.ascontiguousarray(qr, dtype=np.float64)
    D = C.c_double()
    i = lib().orc_nn_config(n, d, _dptr(x), _dptr(qr), C.byref(D))
    return i, D.value


def publish_winner(U, C_, w):
    """Index of the lexicographic minimum (U, C, worker) of successful bridges."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    C_ = np.ascontiguousarray(C_, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.int32)
    return lib().orc_publish_winner(len(U), _dptr(U), _dptr(C_), w.ctypes.data_as(_I))


def bridge(prob, qa, ta, troot_a, cost_a, forward, x, troot, cost, seg, U0, C0, res):
    """One bridge step of node a against candidate rows x [n][d+1]: returns
    (ok, candidate group or -1, candidate index, improves, validated, U, C)."""
    h = _ProblemHandle(prob)
    qa = np.ascontiguousarray(qa, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    troot = np.ascontiguousarray(troot, dtype=np.float64)
    cost = np.ascontiguousarray(cost, dtype=np.float64)
    seg = np.ascontiguousarray(seg if seg is not None else np.zeros(len(x)), dtype=np.int32)
    out = np.zeros(4, dtype=np.int32)
    od = np.zeros(2)
    ok = lib().orc_bridge(h.ref, _dptr(qa), float(ta), float(troot_a), float(cost_a), 1 if forward else 0, len(x),
                          _dptr(x), _dptr(troot), _dptr(cost), seg.ctypes.data_as(_I), float(U0), float(C0),
                          float(res), out.ctypes.data_as(_I), _dptr(od))
    return bool(ok), int(out[0]), int(out[1]), bool(out[2]), int(out[3]), od[0], od[1]
