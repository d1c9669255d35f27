"""The oracle's rest frame against the worked examples the paper prints.

For every example in ``tests/golden/paper_examples.txt`` the oracle derives the rest frame
(gamma0, beta0, Sec. "Lorentz Transformation") and the rest-frame resonant wavenumber k*
(static: gamma0 beta0 k_u; optical: gamma0 (1 + beta0) k_L); the lab resonant wavelength it
implies, 2 pi / (k* gamma0 (1 + beta0)), must fall in the interval the printed value stands for.
A dropped (1 + K^2/2), a planar/helical or static/optical mix-up, or a missing Doppler factor
moves it far outside.
"""
import math
import os

import pytest

import oracle
import workloads

HERE = os.path.dirname(os.path.abspath(__file__))


def _examples():
    rows = []
    with open(os.path.join(HERE, "golden", "paper_examples.txt")) as f:
        for line in f:
            if not line.strip() or line.lstrip().startswith("#"):
                continue
            p = line.split(None, 8)
            rows.append(dict(name=p[0], kind=int(p[1]), gamma=float(p[2]), K=float(p[3]), lam=float(p[4]),
                             printed=float(p[5]), lo=float(p[6]), hi=float(p[7]), cite=p[8].strip()))
    return rows


EXAMPLES = _examples()


def test_fixture_is_complete():
    assert len(EXAMPLES) == 6
    for e in EXAMPLES:
        assert e["lo"] <= e["printed"] <= e["hi"] and e["cite"]


@pytest.mark.parametrize("ex", EXAMPLES, ids=[e["name"] for e in EXAMPLES])
def test_resonance_of_paper_examples(ex):
    base = workloads.WORKLOADS["undulator_24x24x96"]
    w = workloads.scaled(base, und_kind=ex["kind"], gamma=ex["gamma"], K=ex["K"], lambda_u=ex["lam"],
                         n_periods=10 if ex["kind"] < 2 else 0, waist=0.0, n_particles=0)
    r = oracle.Run(oracle.params_from(w))
    info = r.info()
    r.close()
    lam = 2.0 * math.pi / (info["kstar"] * info["gamma0"] * (1.0 + info["beta0"]))
    assert ex["lo"] <= lam <= ex["hi"], (ex["name"], lam, ex["printed"])


def test_optical_equivalence_stated_in_example3():
    """Example 3 states that a0 = K and lambda_L = 2 lambda_u reproduce a static undulator's
    resonance: the oracle's rest frames must then agree (to the 1/gamma^2 terms)."""
    base = workloads.WORKLOADS["undulator_24x24x96"]
    out = []
    for kind, lam in ((0, 3.0e-2), (2, 6.0e-2)):
        w = workloads.scaled(base, und_kind=kind, gamma=100.41, K=1.417, lambda_u=lam,
                             n_periods=10 if kind == 0 else 0, waist=0.0, n_particles=0)
        r = oracle.Run(oracle.params_from(w))
        i = r.info()
        r.close()
        out.append((i["gamma0"], 2.0 * math.pi / (i["kstar"] * i["gamma0"] * (1.0 + i["beta0"]))))
    assert abs(out[0][0] - out[1][0]) < 1e-12 * out[0][0]
    assert abs(out[0][1] - out[1][1]) < 2.0 / 100.41 ** 2 * out[0][1]
