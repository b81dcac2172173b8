"""Pins of the oracle's posterior-predictive simulation (Sec. 4.2: the
learned samples simulated from day zero over the training window and the
days ahead, median and central 99% range per day): with all weight on one
particle, the order statistics equal numpy's inverted-CDF quantiles of the
R trajectories the oracle simulator gives for that particle with the
PREDICT_SIM stream; R = 1 returns that trajectory itself."""
import numpy as np

import oracle as O

Q = [0.005, 0.5, 0.995]


def _model(T=40):
    return O.OracleModel(T=T, P=200_000, A0=20, seed=12)


def _trajectories(m, ua, R, days):
    mm = O.OracleModel(T=days, P=200_000, A0=20, seed=12)
    u = np.repeat(ua[:, None], R, axis=1)
    _, tr = O.simulate(mm, u, c1=0, tag=O.TAG_PREDICT_SIM, traj=True)
    return tr  # [days + 1][6][R]


def test_one_particle_quantiles_match_numpy():
    m = _model()
    u = O.prior(m, 50)
    W = np.zeros(50)
    W[17] = 1.0
    R, days = 501, 55
    out = O.predict(m, u, W, R, days, Q)
    tr = _trajectories(m, u[:, 17], R, days)
    for c, series in enumerate((2, 3, 4)):
        want = np.quantile(tr[:, series, :], Q, axis=1, method="inverted_cdf").T
        assert np.array_equal(out[:, c, :], want.astype(np.int32))
    assert np.all(out[:, :, 0] <= out[:, :, 1]) and np.all(out[:, :, 1] <= out[:, :, 2])


def test_single_draw_is_its_trajectory():
    m = _model()
    u = O.prior(m, 8)
    W = np.eye(8)[3]
    out = O.predict(m, u, W, 1, 30, Q)
    tr = _trajectories(m, u[:, 3], 1, 30)
    for q in range(3):
        assert np.array_equal(out[:, :, q], tr[:, 2:5, 0])


def test_day_zero_is_the_initial_state_and_weights_matter():
    m = _model()
    u = O.prior(m, 200)
    out = O.predict(m, u, None, 400, 60, Q)
    assert np.all(out[0, 0, :] == 20) and np.all(out[0, 1:, :] == 0)
    # two different one-hot weightings give different predictive bands
    a = O.predict(m, u, np.eye(200)[5], 400, 60, Q)
    b = O.predict(m, u, np.eye(200)[150], 400, 60, Q)
    assert not np.array_equal(a, b)
