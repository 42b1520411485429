"""The l(t) surrogate end to end (needs a GPU): data from the batched LB, training
by the project's kernels, held-out error against the LB, gain over Washburn's
law, and the LB fallback above the 2 % ensemble spread."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import surrogate as S  # noqa: E402


@pytest.fixture(scope="module")
def data():
    train = S.surrogate_sweep(11, 192)
    test = S.surrogate_sweep(12, 48)
    return train, S.run_lb(train)["l"], test, S.run_lb(test)["l"]


def test_surrogate_beats_washburn_and_meets_its_bar(data):
    train, l_train, test, l_test = data
    sur = S.Surrogate(members=5, seed=1)
    losses = sur.fit(S.features(train), l_train, steps=2500)
    assert np.all(np.isfinite(losses))
    pred, spread = sur.predict(S.features(test))
    rms = S.rms_rel(pred, l_test)
    wash = S.rms_rel(S.washburn(test), l_test)
    print(f"surrogate RMS {rms:.4f}, Washburn RMS {wash:.4f}, max spread {spread.max():.4f}")
    assert rms < 0.03 and rms < 0.1 * wash
    # the ensemble spread flags the worst queries: error where the spread is small stays small
    ok = spread.max(1) <= 0.02
    if ok.any():
        assert S.rms_rel(pred[ok], l_test[ok]) < 0.03
    sur.close()


def test_fallback_answers_uncertain_queries_with_the_lb(data):
    train, l_train, test, l_test = data
    sur = S.Surrogate(members=3, seed=2)
    sur.fit(S.features(train[:64]), l_train[:64], steps=300)     # deliberately under-trained
    l, bad = S.predict_with_fallback(sur, test[:12], threshold=0.02)
    pred, spread = sur.predict(S.features(test[:12]))
    np.testing.assert_array_equal(np.sort(bad), np.where(spread.max(1) > 0.02)[0])
    assert len(bad) > 0
    # fallback rows are the LB's own l(t), the others the surrogate's
    np.testing.assert_allclose(l[bad], l_test[bad], rtol=1e-12)
    keep = np.setdiff1d(np.arange(12), bad)
    np.testing.assert_allclose(l[keep], pred[keep], rtol=1e-6)
    sur.close()
