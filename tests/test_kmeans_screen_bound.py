"""The error bound behind the FP32 screen of the k-means assignment.

The CUDA assignment computes every squared distance in FP32 and accepts the
FP32 winner only when it is separated from every other centre by more than
the sum of the two distances' error bounds E; otherwise the row runs the
FP64 loop.  That is sound when |d32 - d64| <= E/2 for every row and centre
(E carries a factor 2 of margin), d64 being the FP64 distance with one
rounding per operation (the oracle's).  numpy's float32 and float64 scalar
operations round once each, so they reproduce both computations (the FP32
sum without fused multiply-add, whose error the bound also covers)."""
import numpy as np
import pytest

U = np.float32(2.0 ** -24)


def half_bound(d, nmu, dim):
    """E/2 of the CUDA screen, in float64."""
    u = float(U)
    k_rel = 2.0 * u * (dim + 3) + 2.0 * (dim + 2) * 2.0 ** -53
    return k_rel * d + 2.1 * u * nmu * np.sqrt(d) + 3.0 * u * u * nmu * nmu


def d32_of(x, mu):
    mu32 = mu.astype(np.float32)
    acc = np.float32(0.0)
    for j in range(len(x)):
        t = np.float32(x[j] - mu32[j])
        acc = np.float32(acc + np.float32(t * t))
    return float(acc)


def d64_of(x, mu):
    acc = 0.0
    for j in range(len(x)):
        t = float(np.float64(x[j]) - mu[j])
        acc = acc + t * t
    return acc


@pytest.mark.parametrize("dim", [1, 2, 4, 8, 16])
def test_screen_bound_holds(dim):
    rng = np.random.default_rng(dim)
    worst = 0.0
    for trial in range(3000):
        scale = 10.0 ** rng.uniform(-6, 3)
        mu = rng.standard_normal(dim) * scale
        # rows near the centre (cancellation against a large |mu|), and far
        near = rng.random() < 0.5
        x = (mu + rng.standard_normal(dim) * scale * (1e-4 if near else 1.0)).astype(np.float32)
        d32, d64 = d32_of(x, mu), d64_of(x, mu)
        nmu = float(np.sqrt(np.sum(mu * mu)) * (1 + 1e-6))
        hb = half_bound(d32, nmu, dim)
        assert abs(d32 - d64) <= hb, (trial, d32, d64, hb)
        if hb > 0:
            worst = max(worst, abs(d32 - d64) / hb)
    assert worst < 1.0


@pytest.mark.parametrize("dim", [2, 8, 16])
def test_screen_bound_in_the_subnormal_range(dim):
    """Rows and centres near 1e-21: the FP32 squares and sums fall into the
    subnormal range, where rounding is absolute (at most dim 2^-149 in all),
    and only the bound's 2^-120 floor covers them (the relative terms alone
    would not)."""
    rng = np.random.default_rng(100 + dim)
    floor_needed = False
    for trial in range(3000):
        scale = 10.0 ** rng.uniform(-25, -18)
        mu = rng.standard_normal(dim) * scale
        x = (mu + rng.standard_normal(dim) * scale).astype(np.float32)
        d32, d64 = d32_of(x, mu), d64_of(x, mu)
        nmu = float(np.sqrt(np.sum(mu * mu)) * (1 + 1e-6))
        hb = half_bound(d32, nmu, dim)
        assert abs(d32 - d64) <= hb + 2.0 ** -121, (trial, d32, d64, hb)
        floor_needed |= abs(d32 - d64) > hb
    assert floor_needed  # the case the floor is there for does occur


def test_screen_separates_clear_rows_only():
    """A clearly nearer centre passes the screen; an exact FP64 tie never
    does (the FP64 loop then decides, ties to the smaller centre)."""
    x = np.array([0.5, 0.25, -1.0], dtype=np.float32)
    near = x.astype(np.float64) + 1e-3
    far = x.astype(np.float64) + 1.0
    nmu = lambda m: float(np.sqrt(np.sum(m * m)) * (1 + 1e-6))
    d_near, d_far = d32_of(x, near), d32_of(x, far)
    assert d_near + 2 * half_bound(d_near, nmu(near), 3) < d_far - 2 * half_bound(d_far, nmu(far), 3)
    # two centres mirrored about x: equal FP64 distances
    m1 = x.astype(np.float64) + np.array([0.5, 0.0, 0.0])
    m2 = x.astype(np.float64) - np.array([0.5, 0.0, 0.0])
    assert d64_of(x, m1) == d64_of(x, m2)
    d1, d2 = d32_of(x, m1), d32_of(x, m2)
    assert not (d1 + 2 * half_bound(d1, nmu(m1), 3) < d2 - 2 * half_bound(d2, nmu(m2), 3))
