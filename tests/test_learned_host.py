"""Host logic of the learned-estimator workflow (no GPU): label selection, Philox
key assignment, the procedural scenes' band-smooth scattering, dataset slicing and
the standardisation statistics."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1803_00430_gb300 import learned  # noqa: E402


def test_label_ok_rules():
    p = {
        "rt60_raw": np.array([[0.5, 0.5, 0.5, 0.5, np.nan, 0.01, 40.0, 1.0]]),
        "range_kind": np.array([[1, 2, 3, 1, 1, 1, 1, 0]]),
        "fit_r2": np.array([[0.99, 0.96, 0.99, 0.9, 0.99, 0.99, 0.99, 0.99]]),
    }
    np.testing.assert_array_equal(learned.label_ok(p, 8)[0], [1, 1, 0, 0, 0, 0, 0, 0])


def test_keys_are_distinct():
    lo, (ha, hb) = learned._keys(101, 12)
    keys = lo + [ha, hb]
    assert len(set(keys)) == len(keys)
    lo2, hi2 = learned._keys(202, 12)
    assert not set(keys) & set(lo2 + list(hi2))


def test_learned_scenes_have_band_smooth_scattering():
    for sc in learned.learned_scenes(3, 6):
        s = sc.scattering
        assert np.all(np.diff(s, axis=1) >= -1e-7)
        assert np.all(s.max(axis=1) - s.min(axis=1) <= learned.S_SPREAD + 1e-6)
        assert np.all((s >= 0.1 - 1e-6) & (s <= 0.9 + 1e-6))
        assert sc.num_sources == 1


def _toy(n=10):
    rng = np.random.default_rng(0)
    Y = rng.normal(size=(n, 16)).astype(np.float32)
    M = (rng.uniform(size=(n, 16)) > 0.3).astype(np.float32)
    ref = np.where(M[:, :8] > 0, np.exp(Y[:, :8]), np.nan)
    return learned.Dataset(torch.tensor(rng.normal(size=(n, 528)), dtype=torch.float32), Y, M,
                           ref * 1.1, ref, np.repeat([1000, 2000], n // 2), 5000, 0.7)


def test_dataset_rows_and_normalization():
    ds = _toy()
    sub = ds.rows(ds.rays == 2000)
    assert sub.X.shape == (5, 528) and np.all(sub.rays == 2000)
    np.testing.assert_array_equal(sub.Y, ds.Y[5:])
    np.testing.assert_array_equal(sub.X.numpy(), ds.X.numpy()[5:])
    in_mean, in_std, out_mean, out_std = learned.normalization(ds)
    np.testing.assert_allclose(in_mean, ds.X.double().numpy().mean(axis=0), rtol=1e-12)
    M = ds.mask.astype(bool)
    for j in range(16):
        if M[:, j].sum() > 1:
            assert out_mean[j] == pytest.approx(ds.Y[M[:, j], j].mean(), rel=1e-6)
            assert out_std[j] == pytest.approx(ds.Y[M[:, j], j].std(), rel=1e-6)
