"""Pins of the SVR-RBF oracle (Section 3.4): optimality of the trained
dual, a brute-force QP on a tiny problem, kernel interpolation, the
epsilon tube, the width rounding and the exponential lookup table's bound."""
import numpy as np
import pytest

from oracle import svr


def _problem(n, seed):
    r = np.random.Generator(np.random.PCG64(seed))
    X = r.standard_normal((n, 5))
    # a smooth target of the features plus noise, in the label-index range 0..5
    y = np.clip(2.5 + 1.2 * np.tanh(X[:, 0] - 0.5 * X[:, 2]) + 0.3 * r.standard_normal(n), 0, 5)
    return X, y


def test_fit_meets_the_optimality_conditions():
    X, y = _problem(80, 1)
    # gamma 0.1 (a flat kernel: strongly correlated coordinates) converges slowly
    for C, gamma, eps, tol, cap in ((10.0, 0.1, 0.1, 1e-8, 50000), (1.0, 1.0, 0.25, 1e-10, 10000)):
        m = svr.fit(X, y, C, gamma, eps, tol=tol, max_sweeps=cap)
        assert m["sweeps"] < cap
        assert svr.kkt_violation(m, y, C, eps) <= 1e-7
        # some samples sit inside the tube (beta = 0), some on its edge or at the box
        assert np.any(m["beta"] == 0.0) and np.any(m["beta"] != 0.0)


def test_fit_equals_a_brute_force_qp_on_a_tiny_problem():
    scipy_opt = pytest.importorskip("scipy.optimize")
    X, y = _problem(6, 2)
    C, gamma, eps = 2.0, 0.5, 0.2
    m = svr.fit(X, y, C, gamma, eps, tol=1e-14)
    K1 = svr.rbf(X, X, gamma) + 1.0
    n = len(y)

    # the same dual with beta = p - q, p, q in [0, C]: a smooth bound-constrained QP
    def fun(z):
        b = z[:n] - z[n:]
        g = K1 @ b - y
        val = 0.5 * b @ K1 @ b - y @ b + eps * z.sum()
        return val, np.concatenate([g + eps, -g + eps])

    res = scipy_opt.minimize(fun, np.zeros(2 * n), jac=True, method="L-BFGS-B", bounds=[(0.0, C)] * (2 * n),
                             options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 10000})
    b_qp = res.x[:n] - res.x[n:]
    assert svr.objective(m["beta"], K1, y, eps) <= svr.objective(b_qp, K1, y, eps) + 1e-10
    np.testing.assert_allclose(m["beta"], b_qp, atol=1e-5)


def test_zero_tube_and_open_box_interpolate_the_targets():
    # the Gaussian kernel of distinct points is positive definite: with eps = 0
    # and no box, the optimum solves K1 beta = y and f passes through every target
    X, y = _problem(25, 3)
    m = svr.fit(X, y, C=1e9, gamma=0.3, eps=0.0, tol=1e-13, max_sweeps=200000)
    np.testing.assert_allclose(svr.predict(m, X), y, atol=1e-6)
    K1 = svr.rbf(X, X, 0.3) + 1.0
    np.testing.assert_allclose(m["beta"], np.linalg.solve(K1, y), rtol=1e-5, atol=1e-6)


def test_targets_inside_the_tube_give_the_zero_model():
    X, y = _problem(30, 4)
    m = svr.fit(X, y, C=5.0, gamma=0.2, eps=float(np.abs(y).max()) + 1e-9)
    assert np.all(m["beta"] == 0.0)
    np.testing.assert_array_equal(svr.predict(m, X[:5]), np.zeros(5))


def test_widths_round_up_to_the_next_table():
    f = np.array([-0.3, 0.2, 1.0, 2.5, 4.9, 7.0])
    np.testing.assert_array_equal(svr.widths(f), [4, 6, 6, 12, 0, 0])
    np.testing.assert_array_equal(svr.widths(f, margin=0.25), [4, 4, 6, 12, 0, 0])
    np.testing.assert_array_equal(svr.width_index(np.array([4, 6, 8, 12, 16, 0])), [0, 1, 2, 3, 4, 5])
    np.testing.assert_array_equal(svr.widths(svr.width_index(np.array([8, 0, 4]))), [8, 0, 4])


def test_exp_table_within_its_bound():
    table, step = svr.exp_table(1024, 16.0)
    t = np.linspace(0.0, 20.0, 200001)
    err = np.abs(svr.exp_lut(t, table, step) - np.exp(-t))
    bound = svr.exp_lut_bound(step, 16.0)
    assert err.max() <= bound
    # the interpolation term is what keeps the error small: nearest entries break the bound
    nearest = table[np.clip(np.rint(t / step).astype(np.int64), 0, len(table) - 1)]
    assert np.abs(nearest - np.exp(-t))[t < 16.0].max() > bound


def test_rbf_kernel_values():
    x = np.array([[0.0, 0.0, 0.0, 0.0, 0.0], [1.0, 2.0, 0.0, 0.0, 0.0]])
    K = svr.rbf(x, x, 0.5)
    # |x0 - x1|^2 = 5: exp(-0.5 * 5)
    np.testing.assert_allclose(K, [[1.0, np.exp(-2.5)], [np.exp(-2.5), 1.0]], rtol=0, atol=1e-15)
    y = np.array([[0.0, 0.0, 3.0, 0.0, 4.0]])
    np.testing.assert_allclose(svr.rbf(x[:1], y, 0.1), [[np.exp(-2.5)]], rtol=0, atol=1e-15)


# ------------------------------------------------- the FP32 inference rule

RHO = 1.0 - 2.0 ** -5          # dyadic ratio of the geometric table


def test_geometric_table_is_the_exponential():
    """e_k = rho^k formed by FP64 products equals exp(-k step), step = -ln rho,
    within FP32 rounding plus the products' relative error."""
    tab = svr.exp_table_geometric(1024, RHO)
    step = -np.log(RHO)
    want = np.exp(-np.arange(1024) * step)
    assert np.all(np.abs(tab.astype(np.float64) - want) <= want * (2.0 ** -24 + 1024 * 2.0 ** -52) + 1e-300)
    assert tab[0] == 1.0 and np.all(np.diff(tab) <= 0)


def test_predict32_within_its_error_bound_of_fp64():
    """The FP32 rule with the table exponential stays within the table's
    interpolation bound (step^2/8 + tail) per kernel term, summed over the
    support vectors with their |beta|, plus FP32 rounding of the sum, of the
    FP64 model with the exact exponential."""
    X, y = _problem(120, 5)
    Xn = X.astype(np.float32)
    m = svr.fit(Xn.astype(np.float64), y, 1.0, 1.0, 0.1, max_sweeps=50)
    n, step = 1024, -np.log(RHO)
    tab = svr.exp_table_geometric(n, RHO)
    inv_step = np.float32(1.0 / step)
    beta32 = m["beta"].astype(np.float32)
    r = np.random.Generator(np.random.PCG64(9))
    Xq = r.standard_normal((200, 5)).astype(np.float32)
    f32 = svr.predict32(Xn, beta32, 1.0, inv_step, tab, Xq).astype(np.float64)
    f64 = svr.predict({"X": Xn.astype(np.float64), "beta": beta32.astype(np.float64), "gamma": 1.0}, Xq)
    ab = np.abs(beta32.astype(np.float64)).sum()
    # interpolation + tail + the argument's FP32 roundings (relative 4u of t,
    # so exp changes by at most 4u t e^-t <= 4u/e) + the table's rounding
    per_term = step * step / 8 + np.exp(-(n - 1) * step) + 4 * 2.0 ** -24 + 2 * 2.0 ** -24
    bound = ab * per_term + len(beta32) * 2.0 ** -24 * (ab * 2 + np.abs(f64).max()) * 1.01
    assert np.all(np.abs(f32 - f64) <= bound)
    assert np.abs(f32 - f64).max() > 0          # the rule is not the FP64 model itself


def test_predict32_far_from_every_support_vector_is_the_bias_sum():
    """Past the table every kernel term is exactly 0, so f = fl32 sum of beta_i."""
    sv = np.zeros((3, 5), np.float32)
    beta = np.array([0.5, -0.25, 2.0], np.float32)
    tab = svr.exp_table_geometric(64, RHO)
    f = svr.predict32(sv, beta, 1.0, 1.0 / -np.log(RHO), tab, np.full((1, 5), 100.0, np.float32))
    assert f[0] == np.float32(2.25)
    # at a support vector itself (t = 0) the term is exactly 2 beta
    f0 = svr.predict32(sv[:1], beta[:1], 1.0, 1.0 / -np.log(RHO), tab, sv[:1])
    assert f0[0] == np.float32(1.0)


def test_widths32_round_up_rule():
    f = np.array([-0.5, 0.0, 0.2, 1.0, 2.4, 4.01, 9.0], np.float32)
    np.testing.assert_array_equal(svr.widths32(f, 0.0), [4, 4, 6, 6, 12, 0, 0])
    np.testing.assert_array_equal(svr.widths32(f, 0.5), [4, 4, 4, 6, 8, 16, 0])
