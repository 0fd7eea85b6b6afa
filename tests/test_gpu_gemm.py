"""The tensor-core BF16 GEMM (tcgen05, TMA, tensor memory) through the C ABI
against float64 products of the same bf16 operands.

Tolerance: each output is a float32 sum of K products of bf16 values (exact in
float32), so |D - ref| <= K * 2^-24 * sum_k |a_k b_k| up to the summation
order; the check uses 4 * K * 2^-24 * (|A| |B|') + 1e-30.  Outputs rounded to
bf16 add half an ulp: 2^-9 relative."""
import numpy as np
import pytest

from tests.gpu_util import lib

pytestmark = pytest.mark.gpu


def _bf16(rng, rows, cols, ld=None, scale=1.0):
    import torch
    ld = cols if ld is None else ld
    t = torch.zeros(rows, ld, dtype=torch.bfloat16)
    t[:, :cols] = torch.from_numpy((scale * rng.standard_normal((rows, cols))).astype(np.float32)).to(torch.bfloat16)
    return t.cuda()


def _ref(A, B, K):
    a = A[:, :K].double().cpu().numpy()
    b = B[:, :K].double().cpu().numpy()
    return a @ b.T, np.abs(a) @ np.abs(b).T


def _bound(absprod, K):
    return 4.0 * K * 2.0 ** -24 * absprod + 1e-30


@pytest.mark.parametrize("M,N,K,lda,ldb", [
    (128, 128, 64, 64, 64),          # one tile, one k-step
    (300, 200, 136, 136, 136),       # ragged in M, N and K
    (129, 257, 1000, 1000, 1000),    # ragged, many k-tiles
    (77, 45, 100, 104, 112),         # leading dimensions larger than K
    (1, 1, 8, 8, 8),                 # smallest
    (512, 384, 4096, 4096, 4096),    # several tiles, long K
])
def test_gemm_matches_float64(M, N, K, lda, ldb):
    import torch
    pd = lib()
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = _bf16(rng, M, K, lda)
    B = _bf16(rng, N, K, ldb)
    D = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    pd.pdqp_gemm_bf16(A, B, D_f32=D, K=K)
    assert pd.pdqp_gemm_bf16_check() == 0
    ref, absprod = _ref(A, B, K)
    err = np.abs(D.double().cpu().numpy() - ref)
    assert np.all(err <= _bound(absprod, K)), float(np.max(err / _bound(absprod, K)))


@pytest.mark.parametrize("splits", [0, 2, 3, 7])
def test_split_k_matches_unsplit(splits):
    import torch
    pd = lib()
    rng = np.random.default_rng(splits)
    M, N, K = 200, 136, 3000
    A = _bf16(rng, M, K)
    B = _bf16(rng, N, K)
    ws = torch.zeros(16 * M * N, dtype=torch.float32, device="cuda")
    D = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    used = pd.pdqp_gemm_bf16_splits(M, N, K, splits)
    assert used >= 1 and (splits == 0 or used <= splits)
    pd.pdqp_gemm_bf16(A, B, D_f32=D, splits=splits, workspace=ws)
    assert pd.pdqp_gemm_bf16_check() == 0
    ref, absprod = _ref(A, B, K)
    err = np.abs(D.double().cpu().numpy() - ref)
    assert np.all(err <= _bound(absprod, K))


def test_epilogue_bias_relu_bf16_and_mask():
    import torch
    pd = lib()
    rng = np.random.default_rng(5)
    M, N, K = 250, 190, 320
    A = _bf16(rng, M, K)
    B = _bf16(rng, N, K)
    bias = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).cuda()
    ref, absprod = _ref(A, B, K)
    z = ref + bias.double().cpu().numpy()
    # bias + relu, bf16 and float32 outputs at once (ldd a multiple of 8)
    Db = torch.zeros((M, 192), dtype=torch.bfloat16, device="cuda")
    Df = torch.zeros((M, 192), dtype=torch.float32, device="cuda")
    pd.pdqp_gemm_bf16(A, B, bias=bias, relu=True, D_f32=Df, D_bf16=Db)
    assert pd.pdqp_gemm_bf16_check() == 0
    want = np.maximum(z, 0.0)
    tol = _bound(absprod, K) + 1e-6 * np.abs(z)
    got_f = Df[:, :N].double().cpu().numpy()
    assert np.all(np.abs(got_f - want) <= tol)
    got_b = Db[:, :N].double().cpu().numpy()
    assert np.all(np.abs(got_b - want) <= tol + 2.0 ** -8 * np.abs(want))
    # mask: keep where the bf16 mask is > 0
    mask = _bf16(rng, M, N, 192)
    Dm = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    pd.pdqp_gemm_bf16(A, B, mask=mask, D_f32=Dm)
    assert pd.pdqp_gemm_bf16_check() == 0
    keep = mask[:, :N].double().cpu().numpy() > 0
    want = np.where(keep, ref, 0.0)
    assert np.all(np.abs(Dm.double().cpu().numpy() - want) <= _bound(absprod, K))
    assert np.all(Dm.cpu().numpy()[~keep] == 0.0)


def test_large_square_sampled():
    import torch
    pd = lib()
    M = N = K = 4096
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    pd.pdqp_gemm_bf16(A, B, D_f32=D)
    assert pd.pdqp_gemm_bf16_check() == 0
    rng = np.random.default_rng(0)
    rows = rng.integers(0, M, 64)
    a = A[rows].double().cpu().numpy()
    b = B.double().cpu().numpy()
    ref = a @ b.T
    err = np.abs(D[rows].double().cpu().numpy() - ref)
    assert np.all(err <= _bound(np.abs(a) @ np.abs(b).T, K))


def test_invalid_arguments_are_rejected():
    import torch
    pd = lib()
    A = torch.zeros((16, 20), dtype=torch.bfloat16, device="cuda")     # lda = 20: not a multiple of 8
    B = torch.zeros((16, 24), dtype=torch.bfloat16, device="cuda")
    D = torch.zeros((16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(pd.PdqpError):
        pd.pdqp_gemm_bf16(A, B, D_f32=D, K=16)
    with pytest.raises(pd.PdqpError):
        pd.pdqp_gemm_bf16(B, B, D_f32=D, K=32)                           # K > lda
    Ah = torch.zeros((16, 24), dtype=torch.bfloat16)                     # host tensor
    with pytest.raises(pd.PdqpError):
        pd.pdqp_gemm_bf16(Ah, B, D_f32=D, K=16)
    assert pd.pdqp_gemm_bf16_check() == 0


def test_a_wait_that_runs_out_reports_device_timeout_and_the_device_stays_usable():
    """The failure path of the tensor-core kernels, made safely: their bounded
    wait on an mbarrier that nothing completes gives up after 0.2 s, the host
    reads PDQP_DEVICE_TIMEOUT, the flag is cleared and the next GEMM is right."""
    import time

    import torch
    pd = lib()
    t = time.perf_counter()
    st = pd.pdqp_gemm_bf16_wait_probe()
    dt = time.perf_counter() - t
    assert st == pd.PDQP_DEVICE_TIMEOUT
    assert 0.15 <= dt < 10.0
    assert pd.pdqp_gemm_bf16_check() == pd.PDQP_OK
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(256, 128, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(256, 128, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.zeros(256, 256, dtype=torch.float32, device="cuda")
    pd.pdqp_gemm_bf16(A, B, D_f32=D)
    assert pd.pdqp_gemm_bf16_check() == pd.PDQP_OK
    ref = A.double() @ B.double().T
    bound = 4 * 128 * 2.0 ** -24 * (A.double().abs() @ B.double().abs().T)
    assert bool(((D.double() - ref).abs() <= bound + 1e-30).all())
