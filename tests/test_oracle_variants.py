"""Pins of the oracle's variants of the partial ADMM (no GPU).

* Tikhonov warm start, Eqs. (ini_x)-(ini_z): with every pixel observed one
  step is the ridge solution (T^T T + tau I)^{-1} T^T y (dense solve); the
  iteration is an alternating minimisation, so f(x,z) + tau/2 ||x||^2 never
  increases; its fixed point is the masked ridge solution
  (T^T S_y S_y^T T + tau I)^{-1} T^T S_y y_o (dense solve).
* BGS passes (Sec. II-C): many passes with relax = 1 solve the joint x/z
  problem of Eq. (admm_xz_1a) exactly (dense solve); b passes are b
  repetitions of the x- and z-steps with v and d held fixed.
* Penalty adaptation, Eq. (varying_penalty): the recorded penalties follow
  the rule from the recorded residual norms; d is rescaled so that mu d is
  unchanged; an unreachable threshold gives the fixed-mu run bit for bit;
  the adapted run reaches the fixed-mu minimiser.
"""
import numpy as np

import oracle
from paper_1602_01410_gb300 import inputs


def small_problem(seed=0, M=10, N=11, K=3, frac=0.3, lam=2e-3, mu=5e-2):
    rng = np.random.default_rng(seed)
    b = K // 2
    x = inputs.scene_shapes(rng, M, N)
    h = inputs.psf_gaussian(K, 0.8)
    m = inputs.mask_random_missing(rng, M, N, b, frac)
    y = inputs.observe(rng, x, h, m, 40.0)
    return x, y, m, h, lam, mu


def dense_ops(M, N, h):
    """Dense T~ (circular blur, kernel origin at the centre) and D = [D_h; D_v]."""
    P = M * N
    b = h.shape[0] // 2
    T = np.zeros((P, P))
    for i in range(M):
        for j in range(N):
            for p in range(-b, b + 1):
                for q in range(-b, b + 1):
                    T[i * N + j, ((i - p) % M) * N + (j - q) % N] += h[p + b, q + b]
    E = np.eye(P)
    Dh = np.zeros((P, P))
    Dv = np.zeros((P, P))
    for i in range(M):
        for j in range(N):
            Dh[i * N + j, i * N + (j + 1) % N] += 1
            Dv[i * N + j, ((i + 1) % M) * N + j] += 1
    return T, np.vstack([Dh - E, Dv - E])


# ------------------------------------------------------------- Tikhonov ---

def test_tikhonov_one_step_full_observation_is_ridge():
    rng = np.random.default_rng(1)
    M, N, K, tau = 8, 9, 3, 1e-2
    h = inputs.psf_gaussian(K, 0.9)
    y = rng.random((M, N))
    m = np.ones((M, N), np.uint8)
    yt, x = oracle.tikhonov(y, m, h, 1, tau)
    T, _ = dense_ops(M, N, h)
    want = np.linalg.solve(T.T @ T + tau * np.eye(M * N), T.T @ y.ravel())
    assert np.max(np.abs(x.ravel() - want)) < 1e-10 * np.max(np.abs(want))
    assert np.array_equal(yt, y)


def test_tikhonov_objective_never_increases():
    _, y, m, h, _, _ = small_problem(2, frac=0.4)
    tau = 1e-2
    yt = oracle.init_ytilde(y, m, h.shape[0], round_f32=False)
    F = []
    for _ in range(60):
        yt, x = oracle.tikhonov(yt, m, h, 1, tau)
        r = oracle.conv_circ(x, h) - yt
        F.append(0.5 * np.sum(r * r) + 0.5 * tau * np.sum(x * x))
    F = np.array(F)
    assert np.all(np.diff(F) <= 1e-13 * F[:-1])
    assert F[-1] < F[0]


def test_tikhonov_fixed_point_is_masked_ridge():
    _, y, m, h, _, _ = small_problem(3, M=8, N=9, frac=0.3)
    tau = 0.2
    M, N = y.shape
    yt0 = oracle.init_ytilde(y, m, h.shape[0], round_f32=False)
    yt, x = oracle.tikhonov(yt0, m, h, 4000, tau)
    T, _ = dense_ops(M, N, h)
    obs = m.ravel() != 0
    S = np.eye(M * N)[:, obs]
    want = np.linalg.solve(T.T @ S @ S.T @ T + tau * np.eye(M * N), T.T @ S @ y.ravel()[obs])
    assert np.max(np.abs(x.ravel() - want)) < 1e-9
    t = oracle.conv_circ(x, h)
    assert np.max(np.abs((yt - t)[m == 0])) < 1e-9  # z = M_z H x at the fixed point


def test_warm_start_sets_the_initial_state():
    _, y, m, h, lam, mu = small_problem(4, frac=0.3)
    yt0 = oracle.init_ytilde(y, m, h.shape[0], round_f32=True)
    ytw, xw = oracle.tikhonov(yt0, m, h, 7, 1e-3)
    x, st, _ = oracle.admm(y[None], m[None], h, lam, mu, 0, tikh_iters=7, tikh_tau=1e-3)
    assert np.array_equal(st.yt[0], ytw)
    assert np.array_equal(x[0], xw)
    assert np.array_equal(st.v[0], np.stack(oracle.diff_fwd(xw)))
    assert np.all(st.d == 0)


# ---------------------------------------------------------- BGS passes ---

def random_state(rng, M, N):
    return oracle.State(rng.standard_normal((1, M, N)), 0.1 * rng.standard_normal((1, 2, M, N)),
                        0.1 * rng.standard_normal((1, 2, M, N)))


def test_many_passes_solve_the_joint_x_z_problem():
    _, y, m, h, lam, mu = small_problem(5, M=8, N=9, frac=0.25, mu=0.5)
    M, N = y.shape
    rng = np.random.default_rng(6)
    st = random_state(rng, M, N)
    st.yt[0][m != 0] = y[m != 0]
    x, st1, _ = oracle.admm(y[None], m[None], h, lam, mu, 1, relax=1.0, state=st, passes=3000, round_f32=False)
    T, D = dense_ops(M, N, h)
    obs = m.ravel() != 0
    S = np.eye(M * N)[:, obs]
    w = (st.v[0] - st.d[0]).reshape(2 * M * N)
    want = np.linalg.solve(T.T @ S @ S.T @ T + mu * D.T @ D, T.T @ S @ y.ravel()[obs] + mu * D.T @ w)
    assert np.max(np.abs(x[0].ravel() - want)) < 1e-9 * np.max(np.abs(want))


def test_passes_repeat_the_x_and_z_steps():
    _, y, m, h, lam, mu = small_problem(7, frac=0.3)
    M, N = y.shape
    rng = np.random.default_rng(8)
    st = random_state(rng, M, N)
    st.yt[0][m != 0] = y[m != 0]
    x, st1, _ = oracle.admm(y[None], m[None], h, lam, mu, 1, relax=2.0, state=st, passes=3)
    yt = st.yt[0].copy()
    w = st.v[0] - st.d[0]
    for _ in range(3):
        xk = oracle.solve_x(oracle.conv_circ_adj(yt, h) + mu * oracle.diff_adj(w[0], w[1]), h, mu)
        t = oracle.conv_circ(xk, h)
        yt[m == 0] = 2.0 * t[m == 0] - yt[m == 0]
    assert np.max(np.abs(x[0] - xk)) < 1e-12
    assert np.max(np.abs(st1.yt[0] - yt)) < 1e-12
    a = np.stack(oracle.diff_fwd(xk)) + st.d[0]
    assert np.max(np.abs(st1.v[0] - oracle.vsoft(a, lam / mu))) < 1e-12


def test_proposed_ad_pass_count():
    assert [oracle.passes_ad(K) for K in (3, 5, 9, 13, 21)] == [1, 2, 4, 6, 10]


# ------------------------------------------------- penalty adaptation ---

def test_adaptive_rule_follows_the_residual_norms():
    _, y, m, h, lam, mu = small_problem(9, M=12, N=12, frac=0.3, lam=5e-3)
    n = 80
    x, st, s, mh = oracle.admm(y[None], m[None], h, lam, 20.0, n, stats=True, adapt_t=3.0, mu_hist=True)
    changes = 0
    for i in range(n - 1):
        nd = np.sqrt(s[i, 0])
        nv = np.sqrt(s[i, 2] / mh[i])
        f = 2.0 if nd > 3.0 * nv else (0.5 if nv > 3.0 * nd else 1.0)
        assert mh[i + 1] == f * mh[i]
        changes += f != 1.0
    assert changes >= 2
    assert mh[0] == 20.0


def test_d_rescaled_so_that_mu_d_is_unchanged():
    _, y, m, h, lam, mu = small_problem(10, frac=0.3)
    M, N = y.shape
    rng = np.random.default_rng(11)
    st = random_state(rng, M, N)
    st.yt[0][m != 0] = y[m != 0]
    fired = set()
    for mu0 in (1e-6, 1e-4, 1e-2, 1.0, 1e2, 1e4):
        st.mu = mu0
        _, sf, _ = oracle.admm(y[None], m[None], h, lam, mu0, 1, state=st)
        _, sa, _, mh = oracle.admm(y[None], m[None], h, lam, mu0, 1, state=st, adapt_t=3.0, mu_hist=True)
        fired.add(sa.mu / mu0)
        assert np.array_equal(sa.d * sa.mu, sf.d * mu0)
        assert np.array_equal(sa.yt, sf.yt) and np.array_equal(sa.v, sf.v)
    assert {0.5, 2.0} <= fired  # both branches of the rule were exercised


def test_unreachable_threshold_is_fixed_mu():
    _, y, m, h, lam, mu = small_problem(12, frac=0.3)
    a, sa, _ = oracle.admm(y[None], m[None], h, lam, mu, 30)
    b, sb, _ = oracle.admm(y[None], m[None], h, lam, mu, 30, adapt_t=1e300)
    assert np.array_equal(a, b) and np.array_equal(sa.d, sb.d) and sb.mu == mu


def test_adapted_run_reaches_the_fixed_mu_minimiser():
    _, y, m, h, lam, mu = small_problem(5, M=10, N=10, K=3, frac=0.2, lam=1e-2, mu=2e-2)
    xf, _, _ = oracle.admm(y[None], m[None], h, lam, mu, 30000)
    xa, sa, _, mh = oracle.admm(y[None], m[None], h, lam, 50 * mu, 30000, adapt_t=3.0, mu_hist=True)
    assert np.sqrt(np.mean((xa - xf) ** 2)) < 1e-7
