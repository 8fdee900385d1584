"""The identification input train (Section 5.3.1): pulses, then a random-phase
multisine on [0, 2) Hz at 0.05 Hz resolution, each channel independent."""
import numpy as np

from paper_2604_12505_gb300 import workloads as W


def test_train_shape_amplitudes_and_seeding():
    u = W.identification_train(seed=3)
    assert u.shape == (2200, 3)
    np.testing.assert_allclose(np.abs(u).max(axis=0), [20.0, 20.0, 2.0], rtol=1e-12)
    np.testing.assert_array_equal(u, W.identification_train(seed=3))
    assert not np.array_equal(u, W.identification_train(seed=4))
    # the channels are drawn independently
    assert not np.allclose(u[:, 0], u[:, 1])


def test_multisine_has_exactly_the_lines_below_2_hz():
    # over one period (1 / 0.05 Hz = 20 s = 400 samples at 0.05 s) the DFT of
    # the multisine segment is flat on k = 1..39 and zero at DC and above 2 Hz
    u = W.identification_train(seed=5)
    n_pulse = int(round(0.25 * 2200))
    for ch in range(3):
        X = np.abs(np.fft.rfft(u[n_pulse:n_pulse + 400, ch]))
        lines = X[1:40]
        np.testing.assert_allclose(lines, lines.mean(), rtol=1e-9)
        assert X[0] <= 1e-9 * lines.mean()
        assert X[40:].max() <= 1e-9 * lines.mean()
        # and the segment repeats with that period
        np.testing.assert_allclose(u[n_pulse + 400:n_pulse + 800, ch], u[n_pulse:n_pulse + 400, ch],
                                   atol=1e-9 * np.abs(u[:, ch]).max())


def test_pulses_are_rectangular_and_separated_by_rests():
    u = W.identification_train(seed=7)
    n_pulse = int(round(0.25 * 2200))
    for ch, amp in enumerate((20.0, 20.0, 2.0)):
        p = u[:n_pulse, ch]
        assert set(np.unique(p)) <= {-amp, 0.0, amp}
        on = p != 0.0
        starts = np.flatnonzero(on[1:] & ~on[:-1]) + 1
        assert on[0] and len(starts) >= 5
        # every pulse lasts 0.25-1 s and is followed by at least 1 s of rest
        edges = np.flatnonzero(np.diff(on.astype(int))) + 1
        runs = np.diff(np.concatenate([[0], edges, [n_pulse]]))
        assert runs[0::2][:-1].max() <= 20 and runs[0::2][:-1].min() >= 5
        assert runs[1::2][:-1].min() >= 20


def test_zero_order_hold():
    u = np.arange(12.0).reshape(4, 3)
    out = W.zoh(u, 0.05, 11, 0.02)
    np.testing.assert_array_equal(out[:, 0], [0, 0, 0, 3, 3, 6, 6, 6, 9, 9, 9])


def test_train_scaled_to_a_short_horizon_keeps_the_design():
    from paper_2604_12505_gb300.pipeline import identification_inputs
    K, Ts = 1000, 2e-3
    u = identification_inputs(3, K, Ts, seed0=9)
    assert u.shape == (3, K, 3)
    n_pulse = int(round(0.25 * K))
    # one multisine period spans the segment: 39 equal lines, nothing else
    X = np.abs(np.fft.rfft(u[0, n_pulse:, 2]))
    np.testing.assert_allclose(X[1:40], X[1:40].mean(), rtol=1e-9)
    assert X[40:].max() <= 1e-9 * X[1:40].mean() and X[0] <= 1e-9 * X[1:40].mean()
