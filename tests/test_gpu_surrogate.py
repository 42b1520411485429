"""The l(t) surrogate end to end (needs a GPU): data from the batched LB, training
by the project's kernels, held-out error against the LB, gain over Washburn's
law, and the LB fallback above the 2 % ensemble spread."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_0911_0459_gb300 import surrogate as S  # noqa: E402


DATA = os.path.join(os.path.dirname(S.__file__), "data", "surrogate_data.npz")


@pytest.fixture(scope="module")
def data():
    train = S.surrogate_sweep(11, 192)
    test = S.surrogate_sweep(12, 48)
    return train, S.run_lb(train)["l"], test, S.run_lb(test)["l"]


def test_surrogate_trained_on_fresh_lb_curves_beats_washburn(data):
    """The whole pipeline from nothing: 192 curves generated here by the batched LB, a
    5-member ensemble trained by the project's kernels, 48 held-out curves: the network is
    ten times closer to the LB than Washburn's law, and where its spread is small so is
    its error."""
    train, l_train, test, l_test = data
    sur = S.Surrogate(members=5, seed=1)
    losses = sur.fit(S.features(train), l_train, steps=2500)
    assert np.all(np.isfinite(losses))
    pred, spread = sur.predict(S.features(test))
    rms = S.rms_rel(pred, l_test)
    wash = S.rms_rel(S.washburn(test), l_test)
    print(f"surrogate RMS {rms:.4f}, Washburn RMS {wash:.4f}, max spread {spread.max():.4f}")
    assert rms < 0.1 * wash
    ok = spread.max(1) <= 0.02
    if ok.any():
        assert S.rms_rel(pred[ok], l_test[ok]) < 0.1 * wash
    sur.close()


def test_surrogate_meets_the_two_percent_bar_against_fresh_lb_runs():
    """The 2 % bar: trained on the 4096 LB-generated curves of the training sweep, the
    network's l(t) for 64 held-out queries (the first of the seeded test sweep) is within
    2 % RMS of the LB run here, on this build and GPU.  The stored targets of those queries
    are checked against the same fresh runs (they are the LB's own output, up to FP32
    rounding of another build), so neither side of the comparison rests on stored data."""
    d = np.load(DATA)
    test_caps = S.surrogate_sweep(2, int(d["l_test"].shape[0]))[:64]
    fresh = S.run_lb(test_caps)["l"]
    stored = d["l_test"][:64]
    assert np.abs(fresh - stored).max() <= 1e-3 * np.abs(stored).max()
    sur = S.Surrogate(members=5, seed=0)
    sur.fit(d["x_train"], d["l_train"], steps=6000)
    pred, spread = sur.predict(S.features(test_caps))
    rms = S.rms_rel(pred, fresh)
    wash = S.rms_rel(S.washburn(test_caps), fresh)
    print(f"surrogate RMS vs fresh LB {rms:.5f} (Washburn {wash:.3f}), max spread {spread.max():.4f}")
    assert rms < 0.02 and rms < 0.1 * wash
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
