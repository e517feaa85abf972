"""Host logic of the proposal-network training on CPU, with the tensor-core
network replaced by a fake that records its calls: the initialiser (uniform
weights within 1/sqrt(fan_in), zero biases, the unused output rows zero), the
training loop (a validation split disjoint from the training rows, minibatches
drawn from the training rows only, the parameters of the lowest validation
loss restored at the end) and the chunked mean loss over a set."""
import numpy as np
import pytest

from paper_2609_30533_gb300 import proposal as PR
from paper_2609_30533_gb300 import stp


def test_init_params_layout_and_ranges():
    p = PR.init_params(3)
    assert p.dtype == np.float32 and p.size == stp.MLP_NPARAM
    off = 0
    for name, shape in stp._MLP_SHAPES:
        n = int(np.prod(shape))
        a = p[off:off + n].reshape(shape)
        off += n
        if name.startswith("W"):
            lim = 1.0 / np.sqrt(shape[1])
            assert np.all(np.abs(a) <= lim) and np.std(a) > 0.2 * lim
            if name == "W4":
                assert not np.any(a[152:])
        else:
            assert not np.any(a)
    assert off == p.size
    assert np.array_equal(PR.init_params(3), p) and not np.array_equal(PR.init_params(4), p)


class FakeNet:
    """Parameters are one number; a step adds 1; the loss of a set is a
    scripted function of the parameter (so the best step is known)."""

    def __init__(self, max_batch, val_curve):
        self.max_batch = max_batch
        self.p = 0.0
        self.curve = val_curve
        self.train_rows = []
        self.grad_batches = []

    def get_params(self):
        return np.array([self.p])

    def set_params(self, p):
        self.p = float(p[0])

    def train_step(self, X, T, lr):
        self.train_rows.append(X[:, 0].copy())
        self.p += 1.0
        return 1.0

    def gradients(self, X, T):
        self.grad_batches.append(len(X))
        return self.curve(self.p, X), None


def _data(n):
    X = np.zeros((n, 32), dtype=np.float32)
    X[:, 0] = np.arange(n)
    T = np.zeros((n, stp.MLP_NTGT), dtype=np.float32)
    return X, T


def test_training_restores_the_best_validation_step():
    X, T = _data(100)
    # Validation loss falls until step 60, then rises.
    net = FakeNet(512, lambda p, X: abs(p - 60.0) + 1.0)
    log = PR.train(net, X, T, steps=200, batch=32, lr=1e-3, seed=1, val_frac=0.2, eval_every=20)
    assert log.best_step == 60 and log.best_val == 1.0
    assert net.p == 60.0                                   # parameters of step 60 restored
    assert [k for k, _ in log.val] == list(range(0, 201, 20))
    assert len(log.losses) == 200
    # Minibatches come from the 80 training rows only, never from the 20 held back.
    rows = np.concatenate(net.train_rows).astype(int)
    rng = np.random.default_rng(1)
    held = set(rng.permutation(100)[:20].tolist())
    assert not (set(rows.tolist()) & held) and len(set(rows.tolist())) > 60
    assert all(len(r) == 32 for r in net.train_rows)


def test_small_sets_train_without_validation_and_clip_the_batch():
    X, T = _data(6)
    net = FakeNet(512, lambda p, X: 0.0)
    log = PR.train(net, X, T, steps=5, batch=64, lr=1e-3)
    assert log.val == [(0, float("inf"))] and log.best_step == 0
    assert net.p == 5.0                                    # nothing to restore
    assert all(len(r) == 6 for r in net.train_rows)


def test_loss_is_the_row_weighted_mean_over_chunks():
    X, T = _data(1000)
    # Loss of a chunk = its first row index / 100; chunks of 300 rows.
    net = FakeNet(300, lambda p, X: float(X[0, 0]) / 100.0)
    v = PR.loss(net, X, T)
    assert net.grad_batches == [300, 300, 300, 100]
    assert v == pytest.approx((0 * 300 + 3 * 300 + 6 * 300 + 9 * 100) / 1000)
