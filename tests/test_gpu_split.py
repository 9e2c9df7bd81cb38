"""GPU parity of the split-precision (BF16 digit slices on tcgen05) path.

Tolerances: the split product's error is set by the truncation of each
operand row to s*beta - 1 bits and by the dropped digit pairs, about
s * 2^-(s*beta - 1) relative to sum_k |x_ik||y_kj|.  With the default
s = 7, beta = 7 that is ~2e-14; the tests allow 1e-12 relative Frobenius.
Integer-valued inputs are reproduced bit-exactly (all digit products and
their FP32 sums are exact).  The IsoMP step in split form is held to 1e-10
relative Frobenius per step against the FP64 oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2206_05466_gb300.inputs import vorticity_w0

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2206_05466_gb300 import zeitlin as z  # noqa: E402


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _split_plan(N, **kw):
    return z.Plan(N, z.PRECISION_SPLIT, **kw)


def _gemm(plan, X, Y):
    N = X.shape[0]
    Cd = torch.full((N, N), float("nan"), dtype=torch.complex128, device="cuda")
    z.zt_zgemm_skew(plan, _cuda(X), _cuda(Y), Cd)
    return Cd.cpu().numpy()


def _int_su(N, seed, lim=50):
    rng = np.random.default_rng(seed)
    a = rng.integers(-lim, lim + 1, (N, N)).astype(np.float64)
    b = rng.integers(-lim, lim + 1, (N, N)).astype(np.float64)
    Y = a - a.T + 1j * (b + b.T)          # skew-Hermitian, integer valued
    return Y


@pytest.mark.parametrize("N", [1, 2, 5, 64, 128, 129, 200, 256])
def test_integer_inputs_bit_exact(N):
    rng = np.random.default_rng(N)
    X = rng.integers(-60, 61, (N, N)) + 1j * rng.integers(-60, 61, (N, N))
    Y = _int_su(N, N + 1)
    got = _gemm(_split_plan(N), X, Y)
    want = X @ Y
    assert np.array_equal(got, want), np.abs(got - want).max()


@pytest.mark.parametrize("N", [1, 3, 33, 64, 128, 130, 257, 512])
def test_split_product_accuracy(N):
    rng = np.random.default_rng(7 + N)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    Y = vorticity_w0(N, seed=2)
    got = _gemm(_split_plan(N), X, Y)
    want = X @ Y
    assert _rel(got, want) < 1e-12


@pytest.mark.parametrize("s,beta,eg", [(3, 8, 2), (6, 8, 4), (6, 7, 4), (6, 7, 3), (7, 7, 4), (8, 7, 8), (5, 6, 5)])
def test_split_tunings(s, beta, eg):
    # short exact chunks (beta = 8) force many accumulator drains per tile
    N = 1024
    rng = np.random.default_rng(s * 100 + beta)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    Y = vorticity_w0(N, seed=3)
    got = _gemm(_split_plan(N, slices=s, digit_bits=beta, exact_groups=eg), X, Y)
    want = X @ Y
    bound = 4.0 * s * 2.0 ** (-(s * beta - 1)) * np.sqrt(N)   # loose a-priori bound, relative
    assert _rel(got, want) < max(bound, 1e-13)
    Xi = rng.integers(-60, 61, (N, N)) + 0j
    Yi = _int_su(N, 5)
    assert np.array_equal(_gemm(_split_plan(N, slices=s, digit_bits=beta, exact_groups=eg), Xi, Yi), Xi @ Yi)


def test_split_nonfinite_propagates():
    N = 64
    X = np.ones((N, N), complex)
    X[3, 5] = np.inf
    Y = vorticity_w0(N, seed=1)
    got = _gemm(_split_plan(N), X, Y)
    assert np.all(np.isnan(got[3]))
    assert np.all(np.isfinite(np.delete(got, 3, axis=0)))


def test_isomp_trajectory_split_n64():
    N, h, steps = 64, 0.01, 100
    W0 = vorticity_w0(N, seed=0)
    plan = _split_plan(N)
    Wd = _cuda(W0)
    Wo = W0.copy()
    worst = 0.0
    for n in range(steps):
        z.isomp_step(plan, Wd, h)
        Wo, _ = oracle.isomp_step(Wo, h)
        err = _rel(Wd.cpu().numpy(), Wo)
        worst = max(worst, err)
        assert err <= 1e-10, (n, err)
    print(f"split N=64 worst per-step relative error {worst:.3e}")


def test_isomp_split_n1024_first_steps():
    N, h = 1024, 0.01
    W0 = vorticity_w0(N, seed=0)
    plan = _split_plan(N)
    Wd = _cuda(W0)
    Wo = W0
    for n in range(2):
        info = z.isomp_step(plan, Wd, h)
        Wo, oi = oracle.isomp_step(Wo, h)
        assert info["converged"]
        assert _rel(Wd.cpu().numpy(), Wo) <= 1e-10


def test_autotuner_picks_an_accurate_tuning(tmp_path, monkeypatch):
    from paper_2206_05466_gb300 import autotune

    monkeypatch.setenv("ZEITLIN_TUNE_CACHE", str(tmp_path / "tune.json"))
    res = autotune.autotune(256, target=1e-11)
    assert res["rel_err"] <= 1e-11
    assert all("rel_err" in t for t in res["trials"])
    # the second product's digits: within its error share, and no more than the first's
    g2 = res["gemm2"]
    assert 3 <= res["tuning"]["slices2"] <= res["tuning"]["slices"]
    assert g2["errors"][res["tuning"]["slices2"]] <= g2["bound"]
    again = autotune.autotune(256, target=1e-11)   # served from the cache
    assert again["tuning"] == res["tuning"]


def _band(N, width, seed, skew):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    i = np.arange(N)
    X[np.abs(i[:, None] - i[None, :]) > width] = 0
    if skew:
        X = (X - X.conj().T) / 2
    return X


@pytest.mark.parametrize("N", [300, 1024])
def test_zero_unit_skipping_is_exact(N):
    # Skipping digit-pair tiles that are exactly zero must not change a single bit:
    # decaying matrices (leading digits vanish off the diagonal) and banded ones
    # (whole output tiles without any nonzero unit).
    W = vorticity_w0(N, seed=6)
    P = oracle.stream_solve(W)
    cases = [(P, W), (_band(N, 20, 1, False), _band(N, 20, 2, True)), (W, P)]
    for X, Y in cases:
        dense = _gemm(_split_plan(N, dense=1), X, Y)
        skip = _gemm(_split_plan(N), X, Y)
        assert np.array_equal(dense, skip)
        # rows spanning many orders of magnitude: truncation relative to the row
        # maximum weighs more against the small far entries (autotuner target 1e-11)
        assert _rel(skip, X @ Y) < 1e-11


def test_banded_product_has_zero_far_tiles():
    N = 1024
    X, Y = _band(N, 10, 3, False), _band(N, 10, 4, True)
    got = _gemm(_split_plan(N), X, Y)
    i = np.arange(N)
    far = np.abs(i[:, None] - i[None, :]) > 20
    assert np.all(got[far] == 0)
    assert _rel(got, X @ Y) < 1e-12


@pytest.mark.parametrize("N", [200, 1024])
def test_persistent_kernel_equals_one_tile_per_cta(N):
    # The persistent product kernel (one CTA per SM taking tiles from a ticket
    # counter) runs each tile's arithmetic unchanged: bitwise equal results,
    # for the full product and, through IsoMP steps, the lower-triangle one.
    W = vorticity_w0(N, seed=8)
    P = oracle.stream_solve(W)
    persistent = _gemm(_split_plan(N), P, W)
    one_tile = _gemm(_split_plan(N, no_persistent=1), P, W)
    assert np.array_equal(persistent, one_tile)
    outs = []
    for flag in (0, 1):
        plan = z.Plan(N, z.PRECISION_SPLIT, no_persistent=flag)
        Wd = torch.from_numpy(W.copy()).cuda()
        for _ in range(2):
            z.isomp_step(plan, Wd, 0.01)
        outs.append(Wd.cpu().numpy())
        plan.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("order", [0, 1, 2, 3, 4, 5, 6])
def test_launch_orders_give_identical_products(order):
    # the launch order permutes the tiles, never their arithmetic
    N = 700
    W = vorticity_w0(N, seed=12)
    P = oracle.stream_solve(W)
    base = _gemm(_split_plan(N, slices=6, digit_bits=8, exact_groups=2), P, W)
    got = _gemm(_split_plan(N, slices=6, digit_bits=8, exact_groups=2, tile_order=order), P, W)
    assert np.array_equal(got, base)
    for flag in (0, 1):
        plan = z.Plan(N, z.PRECISION_SPLIT, tile_order=order, no_persistent=flag)
        Wd = torch.from_numpy(W.copy()).cuda()
        z.isomp_step(plan, Wd, 0.01)
        want, _ = oracle.isomp_step(W, 0.01)
        assert _rel(Wd.cpu().numpy(), want) <= 1e-10
        plan.close()


@pytest.mark.parametrize("s2", [3, 4, 5])
def test_second_product_digits_step_matches_oracle(s2):
    # B = Pt A^H with fewer digits (slices2): every step still within the split
    # tolerance of the FP64 oracle (B enters W scaled by h^2/4)
    N, h = 160, 0.01
    W0 = vorticity_w0(N, seed=7)
    plan = z.Plan(N, z.PRECISION_SPLIT, slices=6, digit_bits=8, exact_groups=2, slices2=s2)
    Wd = _cuda(W0)
    Wo = W0.copy()
    for n in range(5):
        info = z.isomp_step(plan, Wd, h)
        Wo, st = oracle.isomp_step(Wo, h)
        assert info["converged"] and abs(info["iters"] - st.iters) <= 1
        err = _rel(Wd.cpu().numpy(), Wo)
        assert err <= 1e-10, (s2, n, err)
    plan.close()


def test_second_product_digits_batched_equals_single():
    N, h = 96, 0.01
    tun = dict(slices=6, digit_bits=8, exact_groups=2, slices2=4)
    W0s = [vorticity_w0(N, seed=30 + k) for k in range(3)]
    single = []
    for W0 in W0s:
        p = z.Plan(N, z.PRECISION_SPLIT, **tun)
        W = _cuda(W0)
        for _ in range(2):
            z.isomp_step(p, W, h)
        single.append(W.cpu().numpy())
        p.close()
    plans = [z.Plan(N, z.PRECISION_SPLIT, **tun) for _ in W0s]
    Ws = [_cuda(W0) for W0 in W0s]
    b = z.Batch(plans, Ws, [h] * len(W0s))
    for _ in range(2):
        rc, _ = b.step()
        assert rc == z.ZT_OK
    for W, want in zip(Ws, single):
        assert np.array_equal(W.cpu().numpy(), want)
    b.close()
    for p in plans:
        p.close()


def test_second_product_digits_error_bound():
    # the leading s2 digits of each operand: a product error near 2^-(beta s2) of the row scales
    N = 256
    rng = np.random.default_rng(3)
    X = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    Y = vorticity_w0(N, seed=5)
    want = X @ Y
    prev = None
    for s in (3, 4, 5, 6):
        got = _gemm(z.Plan(N, z.PRECISION_SPLIT, slices=s, digit_bits=8, exact_groups=2), X, Y)
        e = _rel(got, want)
        assert e < 2.0 ** (-8 * s + 12), (s, e)
        if prev is not None:
            assert e < prev / 16, (s, e, prev)
        prev = e


def test_second_product_kernel_form_is_bitwise_neutral():
    # the second product in the persistent or the one-tile-per-CTA kernel: the same bits
    N, h = 300, 0.01
    W0 = vorticity_w0(N, seed=44)
    outs = []
    for form in (1, 2):
        plan = z.Plan(N, z.PRECISION_SPLIT, slices=6, digit_bits=8, exact_groups=2, no_persistent=1,
                      slices2=4, second_form=form)
        Wd = torch.from_numpy(W0.copy()).cuda()
        for _ in range(2):
            z.isomp_step(plan, Wd, h)
        outs.append(Wd.cpu().numpy())
        plan.close()
    assert np.array_equal(outs[0], outs[1])
