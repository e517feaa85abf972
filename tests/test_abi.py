"""C ABI checks that need no GPU: the library loads, exports every entry point
that include/stp.h declares, validates arguments, and fails loudly (no CPU
fallback) when no CUDA device is present."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as WL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(stp_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_2609_30533_gb300 import build as B
    B.build()
    from paper_2609_30533_gb300 import stp
    return stp.lib()


def test_library_exports_every_declared_symbol(L):
    declared = _declared()
    assert {"stp_create_problem", "stp_plan", "stp_check_edges", "stp_free"} <= declared
    for name in sorted(declared):
        assert hasattr(L, name), name


def test_binding_names_match_header(L):
    from paper_2609_30533_gb300 import stp
    assert set(stp.EXPORTED) == _declared()


def test_status_strings(L):
    from paper_2609_30533_gb300 import stp
    assert stp.status_string(0) == "STP_OK"
    assert stp.status_string(5) == "STP_NO_SOLUTION"


def _params(**kw):
    from paper_2609_30533_gb300 import stp
    base = dict(variant=0, n_roots=4, ext_per_iter=64, max_iters=10, budget_ms=0.0, eta=0.1, edge_res=0.01,
                env_dt=0.02, p_new=0.05, p_guided=0.95, t_max=20.0, seed=0, problem_id=0, precision=0,
                learned=0, capacity=0, iters_per_graph=0, t_offset=0.0, continuous=0, self_collision=0,
                launch_mode=0, persist_ctas=0)
    base.update(kw)
    return stp.StpParams(**base)


def _create(prob, params):
    from paper_2609_30533_gb300 import stp
    keep = []

    def a(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(x)
        return x.ctypes.data_as(C.POINTER(C.c_double))

    robot = stp.StpRobot(prob.dof, 1 if prob.arm else 0, a(prob.dh) if prob.arm else None, a(prob.qlo),
                         a(prob.qhi), len(prob.spheres), a(prob.spheres), prob.vmax)
    obs = stp.StpObstacles(len(prob.obs_r), prob.way.shape[1], a(prob.obs_r), a(prob.way))
    h = C.c_void_p()
    s = stp.lib().stp_create_problem(C.byref(robot), C.byref(obs), a(prob.qs), a(prob.qg), C.byref(params),
                                     C.byref(h))
    return s, h


@pytest.mark.parametrize("bad", [dict(n_roots=0), dict(ext_per_iter=0), dict(variant=7), dict(eta=0.0),
                                 dict(p_new=1.5), dict(precision=2), dict(learned=2), dict(max_iters=0),
                                 dict(t_offset=-1.0), dict(continuous=2), dict(self_collision=1)])
def test_invalid_params_rejected_before_any_device_call(L, bad):
    prob, _ = WL.disc2d(0)
    s, h = _create(prob, _params(**bad))
    assert s == 1 and not h.value


def test_invalid_geometry_rejected(L):
    prob, _ = WL.disc2d(0)
    prob.way[0, 1, 0] = prob.way[0, 0, 0]      # non-increasing waypoint times
    s, _ = _create(prob, _params())
    assert s == 1
    prob, _ = WL.disc2d(0)
    prob.qs = np.array([np.nan, 0.0])
    s, _ = _create(prob, _params())
    assert s == 1


@pytest.mark.parametrize("bad", [dict(n_roots=129), dict(ext_per_iter=8193), dict(variant=-1),
                                 dict(edge_res=0.0), dict(env_dt=-0.02), dict(t_max=0.0), dict(p_guided=-0.1),
                                 dict(capacity=-1), dict(iters_per_graph=-1), dict(t_offset=float("inf")),
                                 dict(launch_mode=3), dict(launch_mode=-1), dict(persist_ctas=-1)])
def test_parameter_limits(L, bad):
    prob, _ = WL.disc2d(0)
    s, h = _create(prob, _params(**bad))
    assert s == 1 and not h.value


def _limit_case(which):
    prob, _ = WL.disc2d(0)
    if which == "dof1":
        prob.dof = 1
    elif which == "point-dof4":
        prob.dof = 4
        prob.qlo, prob.qhi = np.zeros(4), np.ones(4)
        prob.qs, prob.qg = np.full(4, 0.05), np.full(4, 0.95)
    elif which == "spheres65":
        prob.spheres = np.tile(prob.spheres[:1], (65, 1))
    elif which == "spheres0":
        prob.spheres = prob.spheres[:0]
    elif which == "obstacles129":
        prob.obs_r = np.full(129, 0.05)
        prob.way = np.repeat(prob.way[:1], 129, axis=0)
    elif which == "waypoints9":
        t = np.arange(9, dtype=float)
        prob.way = np.zeros((len(prob.obs_r), 9, 4))
        prob.way[:, :, 0] = t
    elif which == "box-inverted":
        prob.qlo, prob.qhi = prob.qhi.copy(), prob.qlo.copy()
    elif which == "radius-negative":
        prob.obs_r = prob.obs_r.copy()
        prob.obs_r[0] = -0.01
    elif which == "sphere-frame":
        prob.spheres = prob.spheres.copy()
        prob.spheres[0, 0] = 1.0            # a point robot has only frame 0
    elif which == "vmax0":
        prob.vmax = 0.0
    return prob


@pytest.mark.parametrize("which", ["dof1", "point-dof4", "spheres65", "spheres0", "obstacles129", "waypoints9",
                                   "box-inverted", "radius-negative", "sphere-frame", "vmax0"])
def test_geometry_limits(L, which):
    s, h = _create(_limit_case(which), _params())
    assert s == 1 and not h.value


def test_null_arguments(L):
    assert L.stp_create_problem(None, None, None, None, None, None) == 1
    assert L.stp_plan(None, None, None, None, None, 0, None) == 1
    assert L.stp_check_edges(None, 0, None, None, None, None, 0, None, None, None) == 1
    L.stp_free(None)
    L.stp_release_cached()     # an empty cache (no device needed)


def test_no_cpu_fallback_without_gpu(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    prob, _ = WL.disc2d(0)
    s, h = _create(prob, _params())
    assert s == 3 and not h.value     # STP_ERR_CUDA


def test_mlp_argument_checks_and_no_cpu_fallback(L):
    h = C.c_void_p()
    assert L.stp_mlp_create(0, C.byref(h)) == 1          # STP_ERR_INVALID
    assert L.stp_mlp_create(65537, C.byref(h)) == 1
    assert L.stp_mlp_create(16, None) == 1
    import torch
    if not torch.cuda.is_available():
        assert L.stp_mlp_create(16, C.byref(h)) == 3     # STP_ERR_CUDA: no device, no fallback


def test_selftest_rejects_bad_limits_and_fails_loudly_without_device(L):
    assert L.stp_selftest_bounded_wait(0, None) == 1
    assert L.stp_selftest_bounded_wait(10 ** 11, None) == 1
    import torch
    if not torch.cuda.is_available():
        assert L.stp_selftest_bounded_wait(1000000, None) == 3


def test_continuous_validation_needs_a_point_robot(L):
    prob, _ = WL.ur5e(0)
    s, h = _create(prob, _params(continuous=1))
    assert s == 1 and not h.value
