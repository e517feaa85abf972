"""FP64 reference of the learned proposal network (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU legs may import this
module. The proposal network is the learned sampling branch (Sec. "Learned
proposal" of the method's GPU form): a 4-layer MLP of width 256 maps a
problem summary to a mixture over the normalised arrival time T/H and to 16
space-time waypoints of a likely path.

Layout (shared by the CUDA path through the C ABI, not through code):
  input x[32]   q_s (7, normalised to [-1, 1] per joint, zero padded), q_g (7),
                DOF one-hot (3: d = 2, 6, 7), mean over obstacles of
                (first waypoint x, y, z, mean velocity x, y, z, radius) (7),
                H / 60, L_g / H (2), zero padding (6).
  hidden        h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3)
  output y[160] mixture logits a[0:8], means mu[8:16] (of T/H), log-stds
                s[16:24] (clamped to [-7, 2]), waypoints [24:152] as 16 x
                (q offset (7), t / H), padding [152:160]; the q offset of
                waypoint i is its normalised configuration minus
                (1 - f_i) u_s + f_i u_g, f_i = (i + 1) / 17.
  loss          NLL of tau = U/H under the mixture + masked mean squared error
                of the waypoints (joints beyond d are masked out).
  targets[130]  tau, 16 x 8 waypoint targets, d.

Every function is the plain definition: dense matrix products, explicit
softmax / log-sum-exp, the closed-form mixture gradient, Adam as published
(Kingma and Ba, 2015).
"""
from __future__ import annotations

import math
from typing import Dict, Tuple

import numpy as np

IN, HID, OUT = 32, 256, 160
N_MIX, N_WP, WP_DIM = 8, 16, 8
OUT_USED = 3 * N_MIX + N_WP * WP_DIM  # 152
N_TGT = 1 + N_WP * WP_DIM + 1         # 130
S_MIN, S_MAX = -7.0, 2.0
LAYERS = (("W1", "b1", IN, HID), ("W2", "b2", HID, HID), ("W3", "b3", HID, HID), ("W4", "b4", HID, OUT))


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (round to nearest, ties to even) via FP32, returned as float64."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(rng: np.random.Generator) -> Dict[str, np.ndarray]:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases; W4 rows
    beyond the used outputs are zero."""
    P = {}
    for w, b, fi, fo in LAYERS:
        lim = 1.0 / math.sqrt(fi)
        P[w] = rng.uniform(-lim, lim, size=(fo, fi))
        P[b] = np.zeros(fo)
    P["W4"][OUT_USED:] = 0.0
    return P


def features(prob, H: float) -> np.ndarray:
    """Problem summary x[32] (layout in the module docstring)."""
    d = prob.dof
    lo, hi = np.asarray(prob.qlo, float), np.asarray(prob.qhi, float)
    x = np.zeros(IN)
    x[0:d] = 2.0 * (np.asarray(prob.qs, float) - lo) / (hi - lo) - 1.0
    x[7:7 + d] = 2.0 * (np.asarray(prob.qg, float) - lo) / (hi - lo) - 1.0
    if d == 2:
        x[14] = 1.0
    elif d == 6:
        x[15] = 1.0
    elif d == 7:
        x[16] = 1.0
    way = np.asarray(prob.way, float)  # [M][K][4] (t, x, y, z)
    M, K = way.shape[0], way.shape[1]
    if M > 0:
        feat = np.zeros((M, 7))
        feat[:, 0:3] = way[:, 0, 1:4]
        if K > 1:
            dt = way[:, K - 1, 0] - way[:, 0, 0]
            feat[:, 3:6] = (way[:, K - 1, 1:4] - way[:, 0, 1:4]) / dt[:, None]
        feat[:, 6] = np.asarray(prob.obs_r, float)
        x[17:24] = feat.mean(axis=0)
    D = float(np.linalg.norm(np.asarray(prob.qg, float) - np.asarray(prob.qs, float)))
    x[24] = H / 60.0
    x[25] = D / prob.vmax / H
    return x


def forward(P: Dict[str, np.ndarray], X: np.ndarray, bf16: bool = False):
    """Returns y [B][160] and the cache for backward. bf16=True rounds weights
    and the inputs of every product to bfloat16 (as the tensor-core path does)."""
    r = bf16_round if bf16 else (lambda a: a)
    Ws = {w: r(P[w]) for w, _, _, _ in LAYERS}
    a0 = r(X)
    z1 = a0 @ Ws["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    a1 = r(h1)
    z2 = a1 @ Ws["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    a2 = r(h2)
    z3 = a2 @ Ws["W3"].T + P["b3"]
    h3 = np.maximum(z3, 0.0)
    a3 = r(h3)
    y = a3 @ Ws["W4"].T + P["b4"]
    cache = dict(a0=a0, a1=a1, a2=a2, a3=a3, z1=z1, z2=z2, z3=z3, Ws=Ws)
    return y, cache


def mixture_terms(y: np.ndarray):
    a = y[:, 0:N_MIX]
    mu = y[:, N_MIX:2 * N_MIX]
    s_raw = y[:, 2 * N_MIX:3 * N_MIX]
    s = np.clip(s_raw, S_MIN, S_MAX)
    return a, mu, s, s_raw


def _lse(v: np.ndarray) -> np.ndarray:
    m = v.max(axis=1, keepdims=True)
    return (m + np.log(np.exp(v - m).sum(axis=1, keepdims=True)))[:, 0]


def wp_mask(dof: np.ndarray) -> np.ndarray:
    """[B][16*8] mask: joints j < d and the time entry of every waypoint."""
    B = len(dof)
    m = np.zeros((B, N_WP, WP_DIM))
    for n in range(B):
        m[n, :, :int(dof[n])] = 1.0
        m[n, :, WP_DIM - 1] = 1.0
    return m.reshape(B, N_WP * WP_DIM)


def loss(y: np.ndarray, T: np.ndarray):
    """Per-sample loss and dL/dy for the batch mean loss. T = targets [B][130]."""
    B = y.shape[0]
    tau = T[:, 0]
    tgt = T[:, 1:1 + N_WP * WP_DIM]
    dof = T[:, -1]
    a, mu, s, s_raw = mixture_terms(y)
    sig = np.exp(s)
    z = (tau[:, None] - mu) / sig
    logpi = a - _lse(a)[:, None]
    l = logpi - 0.5 * z * z - s - 0.5 * math.log(2.0 * math.pi)
    nll = -_lse(l)
    gam = np.exp(l - _lse(l)[:, None])          # responsibilities
    pi = np.exp(logpi)
    g_a = pi - gam
    g_mu = -gam * z / sig
    g_s = gam * (1.0 - z * z) * ((s_raw >= S_MIN) & (s_raw <= S_MAX))
    m = wp_mask(dof)
    wp = y[:, 3 * N_MIX:OUT_USED]
    cnt = m.sum(axis=1)
    mse = (m * (wp - tgt) ** 2).sum(axis=1) / cnt
    g_wp = 2.0 * m * (wp - tgt) / cnt[:, None]
    dy = np.zeros_like(y)
    dy[:, 0:N_MIX] = g_a
    dy[:, N_MIX:2 * N_MIX] = g_mu
    dy[:, 2 * N_MIX:3 * N_MIX] = g_s
    dy[:, 3 * N_MIX:OUT_USED] = g_wp
    return nll + mse, dy / B


def backward(P: Dict[str, np.ndarray], cache, dy: np.ndarray, bf16: bool = False):
    """Gradients of sum(dy * y) with respect to every parameter (dy already
    carries the 1/B of the batch mean)."""
    r = bf16_round if bf16 else (lambda a: a)
    Ws = cache["Ws"]
    g = {}
    d = r(dy) if bf16 else dy
    g["W4"] = d.T @ cache["a3"]
    g["b4"] = dy.sum(axis=0)
    dh3 = (d @ Ws["W4"]) * (cache["z3"] > 0)
    d = r(dh3) if bf16 else dh3
    g["W3"] = d.T @ cache["a2"]
    g["b3"] = dh3.sum(axis=0)
    dh2 = (d @ Ws["W3"]) * (cache["z2"] > 0)
    d = r(dh2) if bf16 else dh2
    g["W2"] = d.T @ cache["a1"]
    g["b2"] = dh2.sum(axis=0)
    dh1 = (d @ Ws["W2"]) * (cache["z1"] > 0)
    d = r(dh1) if bf16 else dh1
    g["W1"] = d.T @ cache["a0"]
    g["b1"] = dh1.sum(axis=0)
    return g


def batch_loss(P, X, T) -> float:
    y, _ = forward(P, X)
    return float(loss(y, T)[0].mean())


def adam_init(P):
    return {k: (np.zeros_like(v), np.zeros_like(v)) for k, v in P.items()}


def adam_step(P, G, state, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step counts from 1)."""
    for k in P:
        m, v = state[k]
        m[...] = b1 * m + (1.0 - b1) * G[k]
        v[...] = b2 * v + (1.0 - b2) * G[k] * G[k]
        mh = m / (1.0 - b1 ** step)
        vh = v / (1.0 - b2 ** step)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    P["W4"][OUT_USED:] = 0.0
    P["b4"][OUT_USED:] = 0.0


def path_targets(path: np.ndarray, U: float, H: float, dof: int, lo, hi) -> np.ndarray:
    """targets[130] of a solution path [n][d+1] (q..., t) from q_s = path[0]
    to q_g = path[-1], arriving at U: tau = U/H, and the path sampled at times
    t_i = (i+1) U / 17, i = 0..15, by linear interpolation in t, joints
    normalised to [-1, 1] and taken relative to the straight line
    (1 - f_i) u_s + f_i u_g (f_i = (i+1)/17), time entry t_i / H."""
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    us = 2.0 * (path[0, :dof] - lo) / (hi - lo) - 1.0
    ug = 2.0 * (path[-1, :dof] - lo) / (hi - lo) - 1.0
    t = path[:, dof]
    out = np.zeros(N_TGT)
    out[0] = U / H
    for i in range(N_WP):
        ti = (i + 1) * U / (N_WP + 1)
        k = int(np.searchsorted(t, ti, side="right")) - 1
        k = min(max(k, 0), len(t) - 2)
        f = (ti - t[k]) / (t[k + 1] - t[k])
        q = path[k, :dof] + f * (path[k + 1, :dof] - path[k, :dof])
        o = 1 + i * WP_DIM
        fi = (i + 1) / (N_WP + 1)
        out[o:o + dof] = (2.0 * (q - lo) / (hi - lo) - 1.0) - ((1.0 - fi) * us + fi * ug)
        out[o + WP_DIM - 1] = ti / H
    out[-1] = dof
    return out



# Element-wise tolerance of the tensor-core path (bfloat16 operands, FP32
# accumulation) against forward/backward(..., bf16=True), which round the same
# operands: the two differ by FP32 accumulation order and by activations whose
# FP32 values straddle a bfloat16 rounding boundary (one bfloat16 ulp, at most
# 2^-7 relative). An element passes when
#   |got - ref| <= RTOL * |ref| + RTOL * rms(ref over its slice),
# RTOL = 2 ulps forward (2^-6), 4 ulps backward (2^-5: the backward pass adds
# a rounding of every output gradient). The slice RMS term covers elements
# near zero, where a relative bound is meaningless.
RTOL_FWD = 2.0 ** -6
RTOL_BWD = 2.0 ** -5
# Output slices checked separately: mixture logits, means, log-sds, waypoints, padding.
OUT_SLICES = (("logits", 0, 8), ("means", 8, 16), ("log_sd", 16, 24), ("waypoints", 24, OUT_USED),
              ("padding", OUT_USED, OUT))


def close_elementwise(got: np.ndarray, ref: np.ndarray, rtol: float):
    """(all within tolerance, worst |got - ref| / tolerance) for one slice."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if ref.size == 0:
        return True, 0.0
    scale = float(np.sqrt(np.mean(ref * ref)))
    tol = rtol * np.abs(ref) + rtol * scale + 1e-30
    worst = float(np.max(np.abs(got - ref) / tol))
    return worst <= 1.0, worst
