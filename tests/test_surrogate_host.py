"""Host logic of the learned forward surrogate (no GPU): the geometry channels
and layer table agree with the oracle's, the training models are seeded and
in range, and the FD gate (GatedSurrogate) checks, accepts, falls back and
records as documented -- driven by fake FD and surrogate gradients."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import surrogate as OS  # noqa: E402


@pytest.fixture(scope="module")
def S():
    from paper_2603_16393_gb300 import surrogate
    return surrogate


def test_geometry_and_layers_match_the_oracle(S):
    np.testing.assert_array_equal(S.geometry_channels(70, 70, [0, 17, 34, 52, 69], 128),
                                  OS.geometry_channels(70, 70, [0, 17, 34, 52, 69],
                                                       128).astype(np.float32))
    assert S.layer_table(128, 256, 5120) == OS.layer_table(128, 256, 5120)
    assert S.LAYERS == OS.LAYERS


def test_training_models_are_seeded_and_in_range():
    from paper_2603_16393_gb300 import inputs as I
    a = I.surrogate_training_models(3, 12, 20, 24)
    b = I.surrogate_training_models(3, 12, 20, 24)
    np.testing.assert_array_equal(a, b)
    assert a.min() >= I.V_MIN and a.max() <= I.V_MAX
    # blurring keeps a constant field and the mean of a field (edges replicated)
    c = np.full((9, 11), 2000.0)
    np.testing.assert_allclose(I.blurred_model(c, 2.5), c, rtol=1e-14)


class _FakePlan:
    def __init__(self, g):
        self.g, self.calls = g, 0

    def gradient(self, v, ctx, stream=None):
        self.calls += 1
        return torch.zeros(v.shape[0]), self.g.clone(), None


class _FakeSurrogate:
    def __init__(self, plan, rel):
        self.plan, self.ctx, self.rel, self.calls = plan, None, rel, 0

    def gradient(self, v, stream=None, step=-1):
        self.calls += 1
        return None, self.plan.g * (1.0 + self.rel)


def _rel_cpu(g, ref):
    B = g.shape[0]
    return (g - ref).reshape(B, -1).norm(dim=1) / ref.reshape(B, -1).norm(dim=1)


@pytest.mark.parametrize("rel,threshold", [(0.02, 0.05), (0.08, 0.05)])
def test_gate_checks_accepts_and_falls_back(S, rel, threshold):
    g = torch.ones(3, 4, 5)
    plan = _FakePlan(g)
    sur = _FakeSurrogate(plan, rel)
    gate = S.GatedSurrogate(sur, threshold=threshold, check_every=4, measure=_rel_cpu)
    v = torch.zeros(3, 4, 5)
    used = []
    for step in range(100, 88, -1):
        _, out = gate.gradient(v, step=step)
        used.append("fd" if torch.equal(out, g) else "sur")
    if rel <= threshold:
        # check (FD), three surrogate steps, check, ...
        assert used == ["fd", "sur", "sur", "sur"] * 3
        assert [r.step for r in gate.records] == [100, 96, 92]
        assert all(r.accepted for r in gate.records)
        assert gate.n_surrogate == 9 and gate.n_fd == 3
    else:
        assert used == ["fd"] * 12
        assert len(gate.records) == 1 and not gate.records[0].accepted
        assert gate.rejected and gate.n_fd == 12 and gate.n_surrogate == 0
    assert all(abs(r.error - rel) < 1e-6 for r in gate.records)
