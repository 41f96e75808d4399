"""The tensor-core scoring engine (tcgen05 MMA, TMA, TMEM; three TF32
products per FP32 product) against FP64 on random tiles, including partial
tiles (rows past m/n and K past d are zero-filled by TMA)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,d", [(128, 256, 768), (100, 200, 784), (1, 1, 128), (128, 256, 32), (77, 131, 4)])
def test_tc_tile_matches_fp64(m, n, d):
    import torch
    from paper_2205_00970_b300 import lider
    rng = np.random.default_rng(m * 1000 + n + d)
    A = rng.standard_normal((m, d)).astype(np.float32)
    B = rng.standard_normal((n, d)).astype(np.float32)
    out = lider.tc_tile(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()).cpu().numpy().astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    err = np.abs(out - ref) / scale
    assert np.max(err) < 2e-6, (float(np.max(err)), float(np.mean(err)))


@pytest.mark.parametrize("m,n,d", [(128, 256, 768), (100, 200, 776), (5, 7, 64), (128, 256, 8), (128, 256, 4096)])
def test_tc_tile_f16_accumulation_error(m, n, d):
    """FP16 kind: the products of the FP16-rounded inputs are exact in FP32;
    the tensor cores' FP32 accumulation stays far inside the d * 2^-23 (of the
    absolute sum) that the FP16 guard band allows for it."""
    import torch
    from paper_2205_00970_b300 import lider
    rng = np.random.default_rng(m * 13 + n + d)
    A = rng.standard_normal((m, d)).astype(np.float32)
    B = rng.standard_normal((n, d)).astype(np.float32)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    out = lider.tc_tile(At, Bt, kind=2).cpu().numpy().astype(np.float64)
    A16 = At.half().float().cpu().numpy().astype(np.float64)
    B16 = Bt.half().float().cpu().numpy().astype(np.float64)
    ref = A16 @ B16.T
    scale = np.abs(A16) @ np.abs(B16).T
    err = np.abs(out - ref) / scale
    assert np.max(err) < d * 2.0 ** -23 / 8, (float(np.max(err)), float(np.mean(err)))


@pytest.mark.parametrize("m,n,d", [(128, 256, 768), (100, 200, 784), (5, 7, 64), (128, 256, 16)])
def test_tc_tile_fp8_matches_fp64_of_rounded_inputs(m, n, d):
    """FP8 e4m3 kind (kind::f8f6f4): the products of the e4m3-rounded inputs
    (exact in FP32), accumulated in FP32."""
    import torch
    from paper_2205_00970_b300 import lider
    rng = np.random.default_rng(m * 31 + n + d)
    A = rng.standard_normal((m, d)).astype(np.float32)
    B = rng.standard_normal((n, d)).astype(np.float32)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    out = lider.tc_tile(At, Bt, kind=3).cpu().numpy().astype(np.float64)
    A8 = At.to(torch.float8_e4m3fn).float().cpu().numpy().astype(np.float64)
    B8 = Bt.to(torch.float8_e4m3fn).float().cpu().numpy().astype(np.float64)
    ref = A8 @ B8.T
    scale = np.abs(A8) @ np.abs(B8).T
    err = np.abs(out - ref) / scale
    assert np.max(err) < d * 2.0 ** -23 / 4, (float(np.max(err)), float(np.mean(err)))


@pytest.mark.parametrize("m,n,d", [(128, 256, 768), (100, 200, 776), (5, 7, 64), (128, 256, 8)])
def test_tc_tile_bf16_matches_fp64_of_rounded_inputs(m, n, d):
    """BF16 kind: the products of the BF16-rounded inputs, accumulated in FP32."""
    import torch
    from paper_2205_00970_b300 import lider
    rng = np.random.default_rng(m * 7 + n + d)
    A = rng.standard_normal((m, d)).astype(np.float32)
    B = rng.standard_normal((n, d)).astype(np.float32)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    out = lider.tc_tile(At, Bt, kind=1).cpu().numpy().astype(np.float64)
    A16 = At.to(torch.bfloat16).float().cpu().numpy().astype(np.float64)
    B16 = Bt.to(torch.bfloat16).float().cpu().numpy().astype(np.float64)
    ref = A16 @ B16.T
    scale = np.abs(A16) @ np.abs(B16).T
    err = np.abs(out - ref) / scale
    assert np.max(err) < 3e-5, (float(np.max(err)), float(np.mean(err)))


@pytest.mark.parametrize("kind,d", [(0, 768), (1, 768), (1, 64), (3, 256)])
def test_bounded_wait_runs_out_and_the_device_stays_usable(kind, d):
    """A stage that never fills (the producer leaves it unloaded): the MMA
    warp's wait gives up after its 5 ms limit, the kernel returns on its own
    and the call reports LIDER_ECUDA with the wait's code; the next engine
    call on the same device still gives correct results."""
    import time

    import torch
    from paper_2205_00970_b300 import lider
    rng = np.random.default_rng(d + kind)
    A = torch.from_numpy(rng.standard_normal((128, d)).astype(np.float32)).cuda()
    B = torch.from_numpy(rng.standard_normal((256, d)).astype(np.float32)).cuda()
    t0 = time.perf_counter()
    rc = lider.tc_wait_expiry(A, B, kind=kind, limit_ms=5.0)
    elapsed = time.perf_counter() - t0
    assert rc == -3, rc
    msg = lider.last_error()
    assert "wait timed out (code 2)" in msg, msg           # the full-stage wait of the MMA warp
    assert elapsed < 5.0
    out = lider.tc_tile(A, B, kind=0).cpu().numpy().astype(np.float64)
    ref = A.cpu().numpy().astype(np.float64) @ B.cpu().numpy().astype(np.float64).T
    assert np.max(np.abs(out - ref)) < 1e-3


def _adversarial_rows(rng, m, n, d):
    """Operands that stress FP32 accumulation: terms spanning 2^-8..2^8 in
    magnitude with alternating signs, rows whose second half cancels the
    first exactly, and rows whose products shrink along K (large partial
    sums first, then terms near their rounding unit)."""
    e = rng.integers(-8, 9, size=(m, d)).astype(np.float64)
    A = np.where(rng.random((m, d)) < 0.5, -1.0, 1.0) * np.exp2(e)
    B = np.where(rng.random((n, d)) < 0.5, -1.0, 1.0) * np.exp2(rng.integers(-8, 9, size=(n, d)))
    h = d // 2
    A[: m // 3, h:2 * h] = -A[: m // 3, :h]                  # exact cancellation against equal B halves
    B[: n // 3, h:2 * h] = B[: n // 3, :h]
    decay = np.exp2(-np.floor(np.linspace(0, 16, d)))       # shrinking products along K (powers of two)
    A[m // 3: 2 * m // 3] *= decay
    return A.astype(np.float32), B.astype(np.float32)


@pytest.mark.parametrize("kind", [0, 2], ids=["tf32x3", "f16"])
@pytest.mark.parametrize("m,n,d", [(128, 256, 768), (96, 200, 776)])
def test_tc_tile_accumulation_on_adversarial_operands(kind, m, n, d):
    """The guard bands assume the tensor cores' FP32 accumulation errs by at
    most d 2^-23 of the absolute sum of the products (FP16 kind) and 3e-5 |a|
    |b| (3xTF32, kTcGuard).  Operands built to stress the accumulation
    (cancellation, wide magnitude spread, absorption) stay within them."""
    import torch
    from paper_2205_00970_b300 import lider
    rng = np.random.default_rng(kind * 100 + m + d)
    A, B = _adversarial_rows(rng, m, n, d)
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    out = lider.tc_tile(At, Bt, kind=kind).cpu().numpy().astype(np.float64)
    if kind == 2:
        A64 = At.half().float().cpu().numpy().astype(np.float64)
        B64 = Bt.half().float().cpu().numpy().astype(np.float64)
        assert np.array_equal(A64, A.astype(np.float64)) and np.array_equal(B64, B.astype(np.float64))
        bound = d * 2.0 ** -23 * (np.abs(A64) @ np.abs(B64).T)
    else:
        A64, B64 = A.astype(np.float64), B.astype(np.float64)
        bound = 3e-5 * np.outer(np.linalg.norm(A64, axis=1), np.linalg.norm(B64, axis=1))
    err = np.abs(out - A64 @ B64.T)
    assert np.all(err <= bound), float(np.max(err / bound))
