"""Host logic of the seeded input generators (CPU): the paper's training-data
augmentation (Sec. 4.2) and the flame-vortex field it starts from."""
import numpy as np

from paper_2312_04830_gb300 import workloads as W


def test_augmentation_reduces_to_the_field_samples():
    """With a huge divisor a2 the perturbation a1 (max - min) / a2 vanishes and
    every state is a cell of the field."""
    T, p, Y = W.augmented_field_states(5000, seed=3, grid=16, a2=1e15)
    Tc, pc, Yc = W.flame_vortex_field(16)
    key = {(round(t, 6), tuple(np.round(y, 9))) for t, y in zip(Tc, Yc.T)}
    assert all((round(t, 6), tuple(np.round(y, 9))) in key for t, y in zip(T, Y.T))
    assert np.all(p == pc[0])


def test_augmentation_bounds_and_spread():
    """States stay physical (T in [100, 3500] K, Y in [0, 1] summing to 1);
    the temperature moves by a1 (max T - min T) / a2 with a1 ~ U[-1, 1], so by
    at most span / a2 away from the clipping bounds and by span / (2 a2) on
    average."""
    a2 = 10.0
    T, p, Y = W.augmented_field_states(200000, seed=4, grid=16, a2=a2)
    Tc, _, _ = W.flame_vortex_field(16)
    span = Tc.max() - Tc.min()
    assert T.min() >= 100.0 and T.max() <= 3500.0
    assert Y.min() >= 0.0 and Y.max() <= 1.0
    assert np.allclose(Y.sum(axis=0), 1.0, atol=1e-12)
    rng = np.random.default_rng(4)
    pick = rng.integers(0, Tc.size, T.size)   # the generator's first draw
    dT = T - Tc[pick]
    inside = (Tc[pick] - span / a2 >= 100.0) & (Tc[pick] + span / a2 <= 3500.0)   # never clipped
    assert inside.sum() > 10000
    assert np.abs(dT).max() <= span / a2 * (1 + 1e-12)
    assert abs(np.abs(dT[inside]).mean() / (span / (2 * a2)) - 1) < 0.02


def test_augmentation_is_seeded():
    a = W.augmented_field_states(1000, seed=7, grid=8)
    b = W.augmented_field_states(1000, seed=7, grid=8)
    c = W.augmented_field_states(1000, seed=8, grid=8)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))
    assert not np.array_equal(a[0], c[0])


def test_boxcox_lambda_is_the_maximum_likelihood_exponent():
    """The Box-Cox exponent fitted for Bilger's Z (train.boxcox_lambda)
    against SciPy's maximum-likelihood estimate, and the log-normal case whose
    exponent is 0."""
    import pytest
    ss = pytest.importorskip("scipy.stats")
    from paper_2312_04830_gb300 import train
    rng = np.random.default_rng(0)
    z = rng.beta(0.3, 2.0, 100000)
    assert train.boxcox_lambda(z, 1e-3) == pytest.approx(ss.boxcox_normmax(z + 1e-3, method="mle"), abs=1e-6)
    x = rng.lognormal(0.0, 0.5, 100000)
    assert abs(train.boxcox_lambda(x, 0.0)) < 0.02
