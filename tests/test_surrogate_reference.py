"""The CPU reference of the surrogate network: its analytic gradient is pinned
by central finite differences (FP64), and its BF16 rounding helper by exact cases."""
import numpy as np

from oracle import mlp_reference as ref


def test_bf16_rounding():
    assert ref.bf16(1.0) == 1.0
    assert ref.bf16(1.0 + 2.0 ** -9) == 1.0            # tie -> even
    assert ref.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7
    assert ref.bf16(-3.0) == -3.0
    x = np.random.default_rng(0).normal(size=1000)
    assert np.max(np.abs(ref.bf16(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_reference_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    spec, total = ref.layout()
    flat = rng.normal(0, 0.08, size=total)
    freq = rng.normal(0, 1.0, size=(32, 3))
    pos = rng.normal(0, 2.0, size=(12, 3))
    t = rng.normal(size=12)
    c, inv_r = np.zeros(3), 1.0 / 6.0
    loss, g = ref.loss_and_grad(flat, freq, c, inv_r, pos, t)
    idx = rng.choice(total, 40, replace=False)
    idx = np.concatenate([idx, [total - 1, total - 2]])  # b5, w5
    for i in idx:
        h = 1e-6
        fp = flat.copy()
        fp[i] += h
        fm = flat.copy()
        fm[i] -= h
        lp, _ = ref.loss_and_grad(fp, freq, c, inv_r, pos, t)
        lm, _ = ref.loss_and_grad(fm, freq, c, inv_r, pos, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])
