"""SVR-RBF training in the library (host code, no GPU) against the oracle
(Section 3.4): the same coordinate descent on the same dual, so the same
support weights up to the last bits of exp and of the updates."""
import numpy as np
import pytest

from oracle import svr


@pytest.fixture(scope="module")
def abi():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_07156_gb300 import abi as a
    return a


def _problem(n, seed, dim=5):
    r = np.random.Generator(np.random.PCG64(seed))
    X = r.standard_normal((n, dim))
    y = np.clip(2.5 + 1.2 * np.tanh(X[:, 0] - 0.5 * X[:, -1]) + 0.3 * r.standard_normal(n), 0, 5)
    return X, y


@pytest.mark.parametrize("n,dim,C,gamma,eps", [(64, 5, 1.0, 1.0, 0.25), (200, 5, 10.0, 0.5, 0.1),
                                               (17, 3, 2.0, 2.0, 0.0), (1, 5, 1.0, 1.0, 0.1)])
def test_library_fit_matches_the_oracle(abi, n, dim, C, gamma, eps):
    X, y = _problem(n, 3 + n, dim)
    beta, sweeps = abi.anns_svr_fit(X, y, C, gamma, eps, tol=1e-12, max_sweeps=20000)
    m = svr.fit(X, y, C, gamma, eps, tol=1e-12, max_sweeps=20000)
    np.testing.assert_allclose(beta, m["beta"], rtol=1e-9, atol=1e-9)
    assert abs(sweeps - m["sweeps"]) <= 1
    model = dict(m, beta=beta)
    assert svr.kkt_violation(model, y, C, eps) <= 1e-7


def test_library_fit_argument_errors(abi):
    X, y = _problem(8, 1)
    for args in ((0.0, 1.0, 0.1), (1.0, 0.0, 0.1), (1.0, 1.0, -0.1)):
        with pytest.raises(abi.AnnsError):
            abi.anns_svr_fit(X, y, *args)
    with pytest.raises(abi.AnnsError):
        abi.anns_svr_fit(np.zeros((abi.SVR_MAX_SAMPLES + 1, 2)), np.zeros(abi.SVR_MAX_SAMPLES + 1), 1.0, 1.0, 0.1)
