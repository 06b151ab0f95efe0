"""Pins for the oracle tile rule (CPU only): closed-form spectrum, Weyl bound, hash."""
import numpy as np

from oracle import rsvd, tilerule
from paper_2307_15572_gb300 import synth


def test_noise_hash_symmetric_and_moments():
    rows = np.arange(0, 700)
    cols = np.arange(0, 700)
    e = tilerule.eta(rows, cols, seed=123, scale=1.0)
    assert np.array_equal(e, e.T)
    assert np.all(np.abs(e) <= np.sqrt(3.0))
    v = e[np.triu_indices(700)]
    n = v.size
    assert abs(v.mean()) < 5 * np.sqrt(1.0 / n)
    assert abs((v * v).mean() - 1.0) < 5 * np.sqrt(0.8 / n)   # var(u^2) for U(-sqrt3,sqrt3) = 0.8
    # different seeds give unrelated noise
    e2 = tilerule.eta(rows, cols, seed=124, scale=1.0)
    assert abs(np.corrcoef(e.ravel(), e2.ravel())[0, 1]) < 0.02


def test_mix32_reference_values():
    # lowbias32 is a bijection on 32-bit words with mix(0) = 0
    x = np.arange(1, 1 << 16, dtype=np.uint64)
    h = tilerule.mix32(x)
    assert int(tilerule.mix32(0)) == 0
    assert len(np.unique(h)) == len(x)
    assert np.all(h < (1 << 32))


def _lowbias32_inverse(x):
    # The inverse published with lowbias32 (C. Wellons, hash-prospector):
    # undo the xorshifts and multiply by the modular inverses of the two
    # multipliers (0x846CA68B^-1 = 0x43021123, 0x7FEB352D^-1 = 0x1D69E2A5).
    x = int(x) & 0xFFFFFFFF
    x ^= x >> 16
    x = (x * 0x43021123) & 0xFFFFFFFF
    x ^= (x >> 15) ^ (x >> 30)
    x = (x * 0x1D69E2A5) & 0xFFFFFFFF
    x ^= x >> 16
    return x


def test_mix32_known_answers():
    # Step-by-step trace of the published definition for x = 1:
    #   x ^= x >> 16      -> 0x00000001
    #   x *= 0x7FEB352D   -> 0x7FEB352D
    #   x ^= x >> 15      -> 0x7FEB352D ^ 0x0000FFD6 = 0x7FEBCAFB
    #   x *= 0x846CA68B   -> 0x6889F849   (mod 2^32)
    #   x ^= x >> 16      -> 0x6889F849 ^ 0x00006889 = 0x688990C0
    assert int(tilerule.mix32(1)) == 0x688990C0
    assert int(tilerule.mix32(0x12345678)) == 0xF5E71C96
    assert int(tilerule.mix32(0xFFFFFFFF)) == 0x6768824A
    # the published inverse undoes it on arbitrary words, which fixes both
    # multipliers and all three shifts
    rng = np.random.default_rng(11)
    xs = rng.integers(0, 1 << 32, size=4096, dtype=np.uint64)
    hs = tilerule.mix32(xs)
    assert all(_lowbias32_inverse(h) == int(x) for h, x in zip(hs, xs))
    assert (0x846CA68B * 0x43021123) & 0xFFFFFFFF == 1 and (0x7FEB352D * 0x1D69E2A5) & 0xFFFFFFFF == 1


def test_closed_form_spectrum_matches_dense():
    n, M = 500, 40
    c, s, w = synth.rule_params(M=M, seed=5, decay=8.0)
    A0 = tilerule.dense(n, c, s, w, seed=5, eta_scale=0.0)
    ev_dense = np.sort(np.linalg.eigvalsh(A0))[::-1][:M]
    ev_cf = tilerule.closed_form_eigs(n, c, s, w)
    assert np.max(np.abs(ev_dense - ev_cf)) <= 1e-11 * ev_cf[0]
    assert abs(np.sum(A0 * A0) - tilerule.closed_form_fro2(n, c, s, w)) <= 1e-11 * np.sum(A0 * A0)


def test_weyl_bound_with_noise_and_rsvd():
    n, M = 600, 30
    c, s, w = synth.rule_params(M=M, seed=6, decay=6.0)
    A = tilerule.dense(n, c, s, w, seed=6, eta_scale=1e-7)
    ev_cf = tilerule.closed_form_eigs(n, c, s, w)
    eta_f = np.linalg.norm(A - tilerule.dense(n, c, s, w, seed=6, eta_scale=0.0))
    res = rsvd.rsvd(A, k=M, p=10, q=1, seed=2)
    # A is PSD + tiny symmetric noise: singular values = |eigenvalues|
    big = ev_cf > 1e3 * eta_f
    assert np.all(np.abs(res.S[big] - ev_cf[big]) <= eta_f + 1e-12 * ev_cf[0])


def test_block_equals_dense_submatrix():
    n = 300
    c, s, w = synth.rule_params(M=20, seed=7)
    A = tilerule.dense(n, c, s, w, seed=7, eta_scale=1e-7)
    r = np.arange(50, 90)
    q = np.arange(200, 260)
    assert np.array_equal(tilerule.block(r, q, n, c, s, w, 7, 1e-7), A[np.ix_(r, q)]) or \
        np.allclose(tilerule.block(r, q, n, c, s, w, 7, 1e-7), A[np.ix_(r, q)], rtol=0, atol=1e-15)
