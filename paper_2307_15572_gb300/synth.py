"""Seeded synthetic inputs shaped like the paper's channel matrices.

This module only builds test and benchmark *inputs*; it holds none of the
decomposition's arithmetic and is the one module that both the CUDA path's
tests and the CPU oracle read.  Its random numbers come from numpy's PCG64
(or torch's generator for the GPU-side builder), never from the Philox stream
that defines the sketch matrix.

The paper decomposes dense, symmetric, block-diagonal interaction matrices:
one block per symmetry channel, with channel sizes N = 225 * n_alpha running
from 7650 to 40050 ("Low-rank interactions" paragraph, mesh of 15 x 15
momenta) and singular spectra that fall steeply and then flatten (Fig. 2
discussion).  Those matrix elements are not available here, so these
generators plant a known spectrum instead:

* ``planted_haar``: A = U diag(sigma) U^T with U Haar-distributed (Householder
  QR of a Gaussian matrix, column signs fixed as in Mezzadri, Notices AMS 54,
  2007).  O(n^3): used for n up to a few thousand (the n = 2048 parity case).
* ``planted_mixed``: A = U diag(sigma) U^T with U a product of three rounds of
  (random permutation, random signs, orthonormal Hartley transform).  The
  Hartley matrix H_jk = (cos + sin)(2 pi j k / n) / sqrt(n) is symmetric and
  orthogonal, so U is exactly orthogonal and A has exactly the planted
  spectrum, but building it costs O(n^2 log n) instead of O(n^3).  Used for the
  batched channel set (sizes up to 12,000), where forty Haar matrices would
  take minutes of FP64 QR.
* ``sym_noise``: symmetric Gaussian noise E = s (G + G^T) / sqrt(2).

Sizes, spectra and seeds of the named workloads are listed in ``WORKLOADS``.
"""

import math

import numpy as np

SEED_DENSE = 15572001      # single dense channel, n = 2048
SEED_BATCH = 15572002      # forty uneven channels
SEED_RULE = 15572003       # matrix-free tile rule
SEED_LEARN = 15572004      # learned-rank channel population
SEED_SWEEP = 15572005      # full mixed sweep


def spectrum_exp(n, scale=20.0):
    """sigma_i = exp(-i / scale), i = 1..n."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return np.exp(-i / scale)


def spectrum_pow(n, alpha=2.5):
    """sigma_i = i^-alpha, i = 1..n."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return i ** (-alpha)


def haar_orthogonal(n, rng):
    """Haar-distributed orthogonal n x n matrix (QR of a Gaussian, sign-fixed)."""
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    q *= np.sign(np.diag(r))[None, :]
    return q


def planted_haar(n, sigma, seed):
    """A = U diag(sigma) U^T, U Haar, exactly symmetric, FP64."""
    rng = np.random.default_rng(seed)
    u = haar_orthogonal(n, rng)
    a = (u * sigma[None, :]) @ u.T
    return 0.5 * (a + a.T)


def _hartley_np(m):
    f = np.fft.fft(m, axis=0)
    return (f.real - f.imag) / math.sqrt(m.shape[0])


def _mixing_params(n, rng):
    perms = [rng.permutation(n) for _ in range(3)]
    signs = [rng.choice(np.array([-1.0, 1.0]), size=n) for _ in range(3)]
    return perms, signs


def _apply_mixing_np(m, perms, signs):
    for p, s in zip(perms, signs):
        m = _hartley_np(s[:, None] * m[p, :])
    return m


def planted_mixed(n, sigma, seed, noise_std=0.0):
    """A = U diag(sigma) U^T (+ symmetric noise), U = three Hartley mixing rounds. numpy."""
    rng = np.random.default_rng(seed)
    perms, signs = _mixing_params(n, rng)
    us = _apply_mixing_np(np.diag(sigma), perms, signs)        # U diag(sigma)
    a = _apply_mixing_np(np.ascontiguousarray(us.T), perms, signs)  # U (U diag sigma)^T
    a = 0.5 * (a + a.T)
    if noise_std > 0.0:
        a += sym_noise(n, noise_std, rng)
    return a


def sym_noise(n, std, rng):
    g = rng.standard_normal((n, n))
    return std * (g + g.T) / math.sqrt(2.0)


def planted_mixed_torch(n, sigma, seed, noise_std=0.0, device="cuda"):
    """Same construction as ``planted_mixed`` built with torch on ``device``.

    The permutations and signs come from the same numpy stream, so for a given
    seed this returns the numpy matrix up to FFT rounding (about 1e-15 of
    sigma_1) plus noise drawn from torch's generator (seeded from the same
    seed); use it where only the device copy is needed.
    """
    import torch
    rng = np.random.default_rng(seed)
    perms, signs = _mixing_params(n, rng)
    tp = [torch.as_tensor(p, device=device) for p in perms]
    ts = [torch.as_tensor(s, device=device, dtype=torch.float64) for s in signs]
    scale = 1.0 / math.sqrt(n)

    def apply(m):
        for p, s in zip(tp, ts):
            m = s[:, None] * m[p, :]
            f = torch.fft.fft(m, dim=0)
            m = (f.real - f.imag) * scale
        return m

    sig = torch.as_tensor(sigma, device=device, dtype=torch.float64)
    us = apply(torch.diag(sig))
    a = apply(us.T.contiguous())
    a = 0.5 * (a + a.T)
    if noise_std > 0.0:
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
        e = torch.randn(n, n, device=device, dtype=torch.float64, generator=g)
        a += noise_std * (e + e.T) / math.sqrt(2.0)
    return a.contiguous()


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def dense_case(n=2048, seed=SEED_DENSE):
    """Single dense channel: Haar U, sigma_i = exp(-i/20)."""
    return planted_haar(n, spectrum_exp(n), seed)


def batch_sizes(count=40, lo=1000, hi=12000, seed=SEED_BATCH):
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.integers(lo, hi + 1, size=count)]


def batch_noise_std(n, sigma1=1.0):
    """Entry std giving ||E||_2 ~ 1e-8 sigma_1 (semicircle edge 2 s sqrt(n))."""
    return 1e-8 * sigma1 / (2.0 * math.sqrt(n))


def batch_channel_seed(c, seed=SEED_BATCH):
    return int(np.random.SeedSequence([seed, c]).generate_state(1, dtype=np.uint64)[0])


def batch_channel(c, n, seed=SEED_BATCH, device=None):
    """Channel c of the batched set: sigma_i = i^-2.5, plus noise at 1e-8 sigma_1."""
    sig = spectrum_pow(n, 2.5)
    s = batch_noise_std(n, sig[0])
    cs = batch_channel_seed(c, seed)
    if device is None:
        return planted_mixed(n, sig, cs, s)
    return planted_mixed_torch(n, sig, cs, s, device=device)


def rule_params(M=300, seed=SEED_RULE, decay=25.0):
    """Gaussian-bump tile rule parameters: centres, widths, weights (M each).

    c_m ~ U[0, 8], s_m log-uniform in [0.05, 1.0], w_m = exp(-m / decay).
    """
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.0, 8.0, size=M)
    s = np.exp(rng.uniform(math.log(0.05), math.log(1.0), size=M))
    w = np.exp(-np.arange(1, M + 1, dtype=np.float64) / decay)
    return c, s, w


def learn_channel_params(count=4000, seed=SEED_LEARN, nlo=500, nhi=20000, tlo=1e-7, thi=1e-3):
    """Per-channel (n, tol, rule params) for the learned-rank population.

    Weights mix exponential and algebraic decay,
    w_m = a exp(-m / tau) + (1 - a) m^-beta, a ~ U[0,1], tau ~ logU[5,200],
    beta ~ U[1.5, 4]; tol log-uniform in [tlo, thi] (default [1e-7, 1e-3]);
    M = min(n, 1024) bumps.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nlo, nhi + 1))
        M = min(n, 1024)
        a = rng.uniform()
        tau = math.exp(rng.uniform(math.log(5.0), math.log(200.0)))
        beta = rng.uniform(1.5, 4.0)
        tol = math.exp(rng.uniform(math.log(tlo), math.log(thi)))
        m = np.arange(1, M + 1, dtype=np.float64)
        w = a * np.exp(-m / tau) + (1 - a) * m ** (-beta)
        c = rng.uniform(0.0, 8.0, size=M)
        s = np.exp(rng.uniform(math.log(0.05), math.log(1.0), size=M))
        out.append(dict(n=n, tol=tol, c=c, s=s, w=w,
                        seed=int(rng.integers(0, 2**63 - 1))))
    return out


def sweep_channel_params(count=400, seed=SEED_SWEEP, nlo=2000, nhi=40000, expo=2.41, M=300):
    """Tile-rule channels of the full mixed sweep: sizes drawn from
    p(n) ~ n^-expo on [nlo, nhi] (inverse CDF; expo 2.41 puts the expected
    total of 400 channels at ~150 GB of FP64 entries), each with the
    Gaussian-bump rule's layout (M bumps, centres ~ U[0, 8], widths
    log-uniform in [0.05, 1]) and its own decay w_m = e^{-m / tau},
    tau log-uniform in [10, 50], noise seed and scale 1e-7."""
    rng = np.random.default_rng(seed)
    out = []
    g = 1.0 - expo
    for _ in range(count):
        u = rng.uniform()
        n = int(round((nlo ** g + u * (nhi ** g - nlo ** g)) ** (1.0 / g)))
        tau = math.exp(rng.uniform(math.log(10.0), math.log(50.0)))
        m = np.arange(1, M + 1, dtype=np.float64)
        c = rng.uniform(0.0, 8.0, size=M)
        s = np.exp(rng.uniform(math.log(0.05), math.log(1.0), size=M))
        out.append(dict(n=n, c=c, s=s, w=np.exp(-m / tau), tau=tau, eta=1e-7,
                        seed=int(rng.integers(0, 2**63 - 1))))
    return out


def mixed_decay_spectrum(n, a, tau, beta):
    """sigma_i = a exp(-i / tau) + (1 - a) i^-beta, i = 1..n."""
    i = np.arange(1, n + 1, dtype=np.float64)
    return a * np.exp(-i / tau) + (1.0 - a) * i ** (-beta)


def learn_population(count, seed=SEED_LEARN, nlo=500, nhi=20000, tlo=1e-7, thi=1e-3, tau=(5.0, 200.0),
                     beta=(1.5, 4.0)):
    """Channels for the rank model: sizes uniform in [nlo, nhi], spectra mixing
    exponential and algebraic decay (a ~ U[0,1], tau log-uniform in ``tau``,
    beta uniform in ``beta``; defaults tau ~ logU[5, 200], beta ~ U[1.5, 4]),
    tolerances log-uniform in [tlo, thi]."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(count):
        out.append(dict(n=int(rng.integers(nlo, nhi + 1)), a=float(rng.uniform()),
                        tau=math.exp(rng.uniform(math.log(tau[0]), math.log(tau[1]))),
                        beta=float(rng.uniform(beta[0], beta[1])),
                        tol=math.exp(rng.uniform(math.log(tlo), math.log(thi))),
                        seed=int(rng.integers(0, 2**62))))
    return out


def population_matrix(ch, device=None):
    """Dense planted matrix of one population channel (Hartley-mixed U)."""
    sig = mixed_decay_spectrum(ch["n"], ch["a"], ch["tau"], ch["beta"])
    if device is None:
        return planted_mixed(ch["n"], sig, ch["seed"])
    return planted_mixed_torch(ch["n"], sig, ch["seed"], device=device)


# paper-quoted facts used to size the synthetic channels ("Low-rank
# interactions" paragraph): 15 x 15 momentum mesh, channel sizes 7650..40050.
PAPER_MESH_POINTS = 15 * 15
PAPER_CHANNEL_SIZES = (7650, 40050)

WORKLOADS = {
    "dense2048": dict(n=2048, k=64, p=10, q=2, seed=SEED_DENSE,
                      spectrum="exp(-i/20)", generator="planted_haar"),
    "batch40": dict(count=40, n_range=(1000, 12000), spectrum="i^-2.5",
                    noise="1e-8 sigma_1 spectral", tol=1e-6, metric_tol=1e-4,
                    seed=SEED_BATCH, generator="planted_mixed"),
    "rule200k": dict(n=200000, M=300, k=320, p=10, seed=SEED_RULE),
}
