"""The level-step's wave limiters (Sec. 2.1: phi(theta) a, theta the upwind strength of the same
family over the edge's own) through claw_limiter_eval, the step's own device code, against the
limiter formulas evaluated in IEEE double arithmetic by numpy: minmod, superbee and MC bit for
bit (MC's sum |a| + |b| is formed on the integer pipe and must round exactly like the IEEE sum,
ties to even included), van Leer within four roundings of the exact 2ab / (a + b)."""
import numpy as np
import pytest
import torch

from gpu_helpers import lib_ready

pytestmark = pytest.mark.gpu

NONE, MINMOD, SUPERBEE, VANLEER, MC = 0, 1, 2, 3, 4
TINY = 2.0 ** -1020   # below this the exponent-field halving and doubling are not IEEE operations


@pytest.fixture(scope="module", autouse=True)
def _lib():
    lib_ready()


def _pairs(seed, n=1 << 20):
    """(a, b): random signs; magnitudes over most of the exponent range, pairs of equal and
    nearby magnitudes (frequent rounding ties in the sum), ratios at the branch points of the
    limiters (1/2, 1, 2, 3), zeros and subnormals"""
    rng = np.random.default_rng(seed)
    k = n // 8
    parts = []
    e = rng.uniform(-1000, 1000, k)
    parts.append((2.0 ** e * rng.uniform(1, 2, k), 2.0 ** rng.uniform(-1000, 1000, k)))
    a = 2.0 ** rng.uniform(-900, 900, k) * rng.uniform(1, 2, k)
    parts.append((a, a * rng.uniform(1 / 3.5, 3.5, k)))                 # MC's smooth and doubled branches
    m = rng.integers(1, 1 << 20, k).astype(np.float64)
    parts.append((a, a + m * np.spacing(a)))                            # nearby: the sum's last bit ties
    parts.append((a, a * rng.choice([0.5, 1.0, 2.0, 3.0, 1 / 3.0], k)))  # branch points
    parts.append((a, np.nextafter(3.0 * a, rng.choice([0.0, np.inf], k))))
    sub = rng.integers(1, 1 << 52, k).astype(np.float64) * 2.0 ** -1074
    parts.append((sub, rng.integers(1, 1 << 52, k).astype(np.float64) * 2.0 ** -1074))   # subnormal pairs
    parts.append((a, sub))
    z = np.where(rng.random(k) < 0.5, 0.0, a)
    parts.append((z, np.where(rng.random(k) < 0.5, 0.0, a)))
    A = np.concatenate([p[0] for p in parts])
    B = np.concatenate([p[1] for p in parts])
    A *= rng.choice([-1.0, 1.0], A.size)
    B *= rng.choice([-1.0, 1.0], B.size)
    return A, B


def _device(limiter, A, B):
    from paper_1808_02638_gb300 import claw
    a = torch.from_numpy(A).cuda()
    b = torch.from_numpy(B).cuda()
    out = torch.full_like(a, float("nan"))
    claw.claw_limiter_eval(limiter, a, b, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _want(limiter, A, B):
    ma, mb = np.abs(A), np.abs(B)
    same = (np.signbit(A) == np.signbit(B)) & (ma > 0) & (mb > 0)
    lo, hi = np.minimum(ma, mb), np.maximum(ma, mb)
    if limiter == MINMOD:
        m = lo
    elif limiter == SUPERBEE:
        m = np.maximum(np.minimum(ma, 2 * mb), np.minimum(2 * ma, mb))
    elif limiter == MC:
        with np.errstate(over="ignore"):
            m = np.minimum((ma + mb) * 0.5, 2 * lo)
    else:
        raise ValueError(limiter)
    return np.where(same, np.copysign(m, A), 0.0), same, lo, hi


@pytest.mark.parametrize("limiter", [MINMOD, SUPERBEE, MC])
@pytest.mark.parametrize("seed", [0, 1])
def test_integer_pipe_limiters_equal_the_ieee_formula(limiter, seed):
    A, B = _pairs(seed)
    got = _device(limiter, A, B)
    want, same, lo, hi = _want(limiter, A, B)
    # the formula's halvings and doublings are exact IEEE operations when nothing is subnormal
    # or overflows; that is where the bit patterns must agree
    exact = ~same | ((lo >= TINY) & (hi < 2.0 ** 1022))
    assert exact.mean() > 0.7
    bad = exact & (got.view(np.int64) != want.view(np.int64))
    assert not bad.any(), (A[bad][:4], B[bad][:4], got[bad][:4], want[bad][:4])
    # below 2^-1020 the value may differ from the IEEE evaluation by less than 2^-1020
    rest = ~exact & (hi < 2.0 ** 1022)
    assert np.all(np.abs(got[rest] - want[rest]) < 2.0 ** -1020)


def test_mc_sum_rounds_ties_to_even():
    # |a| + |b| exactly halfway between two doubles: the even neighbour is taken (the sum of the
    # first pair is 2 + 2^-52, halfway between 2 and 2 + 2^-51; MC's value is then the half sum)
    A = np.array([1.0 + 2.0 ** -52, 1.0 + 3 * 2.0 ** -52, 1.5, 2.0 ** 600 * (1 + 2.0 ** -52)])
    B = np.array([1.0, 1.0, 1.5 + 2.0 ** -52, 2.0 ** 600])
    got = _device(MC, A, B)
    want = np.minimum((A + B) * 0.5, 2 * np.minimum(A, B))
    assert np.array_equal(got.view(np.int64), want.view(np.int64))
    assert got[0] == 1.0 and got[1] == 1.0 + 2.0 ** -51


def test_no_limiter_and_van_leer():
    A, B = _pairs(7, 1 << 18)
    assert np.array_equal(_device(NONE, A, B), A)
    got = _device(VANLEER, A, B)
    ma, mb = np.abs(A), np.abs(B)
    same = (np.signbit(A) == np.signbit(B)) & (ma > 0) & (mb > 0)
    ok = same & (ma > 2.0 ** -500) & (mb > 2.0 ** -500) & (ma < 2.0 ** 500) & (mb < 2.0 ** 500)
    # four roundings (the sum, the reciprocal, two products): relative error at most 4 * 2^-53
    # against the exact 2ab / (a + b), checked in rational arithmetic on a sample
    from fractions import Fraction
    idx = np.flatnonzero(ok)[::3]
    worst = Fraction(0)
    for i in idx:
        a, b = Fraction(float(A[i])), Fraction(float(B[i]))
        exact = 2 * a * b / (a + b)
        worst = max(worst, abs(Fraction(float(got[i])) - exact) / abs(exact))
    assert worst <= Fraction(4, 2 ** 53), float(worst) * 2.0 ** 53
    assert np.all(got[~same] == 0.0)


def test_limiter_eval_rejects_bad_arguments():
    from paper_1808_02638_gb300 import claw
    a = torch.zeros(4, dtype=torch.float64, device="cuda")
    for bad in (-1, 5):
        with pytest.raises(claw.ClawError):
            claw.claw_limiter_eval(bad, a, a, a)
    with pytest.raises(ValueError):
        claw.claw_limiter_eval(MC, a, a[:2], a)
