"""The seeded input generator: shapes, determinism and the recipe's structure."""
import numpy as np
import pytest

from paper_1703_06303_gb300 import synth


@pytest.mark.parametrize("cfg", [1, 2])
def test_clip_shapes_and_structure(cfg):
    spec = synth.CONFIGS[cfg]
    clip = synth.make_clip(spec)
    A, W1, mask = clip["A"], clip["W1"], clip["mask"]
    assert A.shape == (spec.m, spec.n) and A.flags.f_contiguous
    assert W1.shape == (spec.m, spec.k) and W1.flags.f_contiguous
    assert np.all(W1 > 0)
    # the first k frames carry no foreground (Section 1: almost pure background)
    assert not mask[:, :spec.k].any()
    assert abs(clip["coverage"] - spec.coverage) <= 0.01 + 1e-12
    again = synth.make_clip(spec)
    assert np.array_equal(A, again["A"]) and np.array_equal(W1, again["W1"])


def test_background_rank_in_weighted_frames():
    spec = synth.CONFIGS[1]
    clip = synth.make_clip(spec)
    s = np.linalg.svd(clip["A"][:, :spec.k], compute_uv=False)
    # rho background directions, the rest at the noise level sigma * sqrt(m)
    assert s[spec.rho - 1] > 10 * s[spec.rho]
    assert s[spec.rho] < 3 * spec.sigma * np.sqrt(spec.m)


def test_batched_specs():
    specs = synth.batched_specs(96)
    assert len(specs) == 96
    assert {s.m for s in specs} <= {4800, 19200, 76800}
    assert all(100 <= s.n <= 800 and 5 <= s.k <= 40 and 3 <= s.r - s.k <= 10 for s in specs)


def test_initial_x1_deterministic():
    a = synth.initial_x1(100, 4, 3)
    assert a.shape == (100, 4) and np.array_equal(a, synth.initial_x1(100, 4, 3))


def test_batched_specs_ranges_and_determinism():
    from paper_1703_06303_gb300 import synth
    a = synth.batched_specs(96)
    b = synth.batched_specs(96)
    assert a == b                                   # same seeds, same workload
    assert len(a) == 96 and len({sp.seed for sp in a}) == 96
    assert {sp.m for sp in a} <= {4800, 19200, 76800}
    for sp in a:
        assert 100 <= sp.n <= 800 and 5 <= sp.k <= 40 and 3 <= sp.r - sp.k <= 10
        assert sp.k <= 64 and sp.r - sp.k <= 32      # within what the library accepts
    assert synth.batched_specs(96, base_seed=7) != a
