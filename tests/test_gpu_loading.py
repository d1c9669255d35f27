"""GPU against the oracle: the quasi-random ellipsoid bunch (Sec. "Electron Bunch Generation")
through mithra_ellipsoid_bunch.  The Halton numbers are rounded operation by operation on both
sides, so the flat part of a uniform profile (z = L (h - 1/2)) is bit-identical; the Gaussian
coordinates go through log / sin / cos / sqrt, whose CUDA and C-library results may differ in
the last bits: 1e-13 relative to each column's scale."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - only on a GPU machine
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2009_13645_gb300 as mithra  # noqa: E402


def _pair(n, **kw):
    eo, eg = oracle.Ellipsoid(), mithra.Ellipsoid()
    for e in (eo, eg):
        e.uniform = kw.get("uniform", 0)
        e.gamma = kw.get("gamma", 100.0)
        for a, v in enumerate(kw.get("sig", (50e-6, 40e-6, 7e-6))):
            e.sig[a] = v
        for a, v in enumerate(kw.get("sig_u", (0.02, 0.03, 0.01))):
            e.sig_u[a] = v
        e.cse_sigma = kw.get("cse_sigma", 0.0)
        e.lambda_r = kw.get("lambda_r", 0.0)
        e.bunching = kw.get("bunching", 0.0)
        e.bunching_phase = kw.get("bunching_phase", 0.0)
        e.shot_noise = kw.get("shot_noise", 0)
        e.charge_e = kw.get("charge_e", 1e9)
    return oracle.ellipsoid_bunch(eo, n), mithra.ellipsoid_bunch(eg, n)


def _close(a, b, tol=1e-13):
    for c in range(6):
        s = max(np.max(np.abs(b[:, c])), 1e-300)
        bound = tol * s
        if c == 5:
            # the spread around sqrt(gamma^2 - 1), plus one rounding of the value itself
            bound = tol * max(np.max(np.abs(b[:, c] - np.mean(b[:, c]))), 1e-300) + 2.3e-16 * s
        assert np.max(np.abs(a[:, c] - b[:, c])) <= bound, c


def test_gaussian_ellipsoid_matches_oracle():
    o, g = _pair(100_003)
    _close(g, o)


def test_uniform_with_edges_bit_identical_flat_part():
    n = 65_536
    o, g = _pair(n, uniform=1, sig=(30e-6, 30e-6, 50e-6), cse_sigma=1.5e-6)
    L = 100e-6
    nu = round(n * L / (L + np.sqrt(2 * np.pi) * 1.5e-6))
    assert np.array_equal(g[:nu, 2], o[:nu, 2])
    _close(g, o)


def test_bunching_and_shot_noise_match_oracle():
    o, g = _pair(200_000, uniform=1, sig=(30e-6, 30e-6, 20e-6), cse_sigma=1e-6, lambda_r=1.0e-6,
                 bunching=0.02, bunching_phase=0.4, shot_noise=1, charge_e=6.2e8)
    _close(g, o, 1e-12)


def test_full_bunch_size_sampled():
    """The FEL run's 2 M particles: every 997th row against the oracle (which computes all)."""
    n = 2_000_000
    o, g = _pair(n, uniform=0, sig=(50e-6, 50e-6, 7e-6), sig_u=(0.02, 0.02, 0.01))
    _close(g[::997], o[::997])


def test_empty_and_rejected():
    e = mithra.Ellipsoid()
    e.gamma = 10.0
    assert mithra.ellipsoid_bunch(e, 0).shape == (0, 6)
    e.gamma = 0.5
    with pytest.raises(mithra.MithraError):
        mithra.ellipsoid_bunch(e, 10)
