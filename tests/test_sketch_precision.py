"""Why the passes over V use two BF16 words (CPU experiment, no GPU).

The range finder is run with V rounded to the word format of each candidate
sketch precision -- FP8 E4M3 with per-tile or per-row scales, one BF16 word,
TF32 (10 stored mantissa bits), two BF16 words -- while the projection uses
the exact V, so only the sketch's precision differs.  At the metric's
tolerance (1e-4, relative Frobenius) on a channel of the batched set
(sigma_i = i^-2.5, l = 128, q = 0, the paper's scheme of Fig. 1), only the
two-word sketch meets the tolerance, at the rank of the FP64 sketch: the
rounding error of a narrower word (relative 2.6e-2, 1.7e-3, 4.1e-4 per
entry) moves the sketched subspace by more than the tolerance.  TF32 meets
it only with one power iteration (two more passes of the same 4 bytes per
entry as two BF16 words), which costs more than the two-word sketch at q = 0.
"""
import numpy as np
import pytest

from paper_2307_15572_gb300 import synth

torch = pytest.importorskip("torch")

N, L, TOL = 2000, 128, 1e-4


def _bf16(x):
    return torch.as_tensor(x).to(torch.bfloat16).to(torch.float64).numpy()


def _tf32(x):
    f = np.asarray(x, dtype=np.float32).view(np.uint32) & np.uint32(0xFFFFE000)
    return f.view(np.float32).astype(np.float64)


def _e4m3(x):
    return torch.as_tensor(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()


def _fp8_tiles(x, t=128):
    out = np.empty_like(x)
    for i in range(0, x.shape[0], t):
        for j in range(0, x.shape[1], t):
            b = x[i:i + t, j:j + t]
            s = np.abs(b).max() / 448.0
            out[i:i + t, j:j + t] = _e4m3(b / s) * s
    return out


def _fp8_rows(x):
    s = np.abs(x).max(axis=1, keepdims=True) / 448.0
    return _e4m3(x / s) * s


@pytest.fixture(scope="module")
def channel():
    A = synth.batch_channel(7, N)
    Om = np.random.default_rng(1).standard_normal((N, L))
    return A, Om


def _run(A, V, Om, q):
    """(k, error): sketch and power passes with V, projection with A."""
    nA = np.linalg.norm(A)
    Q, _ = np.linalg.qr(V @ Om)
    for _ in range(q):
        Q, _ = np.linalg.qr(V @ Q)
        Q, _ = np.linalg.qr(V @ Q)
    u, s, vt = np.linalg.svd(Q.T @ A, full_matrices=False)
    tail = np.sqrt(np.maximum(nA ** 2 - np.cumsum(s ** 2), 0.0)) / nA
    k = int(np.argmax(tail <= TOL)) + 1 if (tail <= TOL).any() else L
    err = np.linalg.norm(A - (Q @ u[:, :k] * s[:k]) @ vt[:k]) / nA
    return k, err


def test_only_two_bf16_words_meet_the_tolerance_without_power_iterations(channel):
    A, Om = channel
    k64, e64 = _run(A, A, Om, 0)
    assert e64 <= TOL and k64 < L
    two = _bf16(A) + _bf16(A - _bf16(A))
    k2, e2 = _run(A, two, Om, 0)
    assert e2 <= TOL and abs(k2 - k64) <= 1
    for V in (_fp8_tiles(A), _fp8_rows(A), _bf16(A), _tf32(A)):
        k, e = _run(A, V, Om, 0)
        assert e > TOL, (k, e)


def test_tf32_needs_a_power_iteration(channel):
    A, Om = channel
    k, e = _run(A, _tf32(A), Om, 1)
    assert e <= TOL and k < L
