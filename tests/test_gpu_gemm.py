"""The surrogate's tensor-core GEMM (tcgen05, TMEM accumulators, TMA for BF16
operands) against an FP64 product of the same BF16-rounded operands.

Every operand path the training pass uses is covered: FP32 operands rounded
while staged and BF16 operands copied by TMA, K-major and MN-major layouts,
batch strides (a zero stride shares an operand), split-K chunks, ragged M, N
and K tails, padded leading dimensions, alpha, beta and bias.  The products
are exact in FP64 up to the kernel's FP32 accumulation, so the bar is the
FP32 summation bound: |C - C_ref| <= 2.4e-7 (k + 4) sum_k |a b| per entry.
"""
import zlib

import pytest

pytestmark = pytest.mark.gpu

# name, M, N, K, batch, kchunk, A bf16, A MN-major, B bf16, B MN-major, alpha, beta, bias, A shared, B shared, pad
CASES = [
    ("f32K x f32MN, K tail 48, bias", 1000, 64, 48, 1, 0, 0, 0, 0, 1, 1.0, 0.0, 1, 0, 0, 0),
    ("bf16K (TMA) x f32MN, K 48, bias", 1000, 64, 48, 1, 0, 1, 0, 0, 1, 1.0, 0.0, 1, 0, 0, 0),
    ("f32K x f32MN, N 128", 1000, 128, 64, 1, 0, 0, 0, 0, 1, 1.0, 0.0, 1, 0, 0, 0),
    ("bf16K x f32MN, residual beta 1", 777, 64, 128, 1, 0, 1, 0, 0, 1, 1.0, 1.0, 1, 0, 0, 0),
    ("shared f32K x f32MN, batch 5, M 96", 96, 64, 128, 5, 0, 0, 0, 0, 1, 1.0, 0.0, 0, 1, 0, 0),
    ("shared f32K x bf16MN (TMA 3-D), batch 5", 128, 64, 96, 5, 0, 0, 0, 1, 1, 1.0, 1.0, 0, 1, 0, 0),
    ("shared f32MN x f32MN, batch 5", 96, 64, 128, 5, 0, 0, 1, 0, 1, 1.0, 0.0, 0, 1, 0, 0),
    ("shared f32MN x bf16MN, batch 5, beta", 128, 64, 96, 5, 0, 0, 1, 1, 1, 1.0, 1.0, 0, 1, 0, 0),
    ("bf16K x f32K, K 16", 1000, 64, 16, 1, 0, 1, 0, 0, 0, 1.0, 0.0, 0, 0, 0, 0),
    ("f32K x f32K, N 128", 1000, 128, 64, 1, 0, 0, 0, 0, 0, 1.0, 0.0, 0, 0, 0, 0),
    ("split-K bf16MN M 48 x f32MN", 48, 64, 5000, 1, 1024, 1, 1, 0, 1, 1.0, 0.0, 0, 0, 0, 0),
    ("split-K bf16MN M 128 x bf16MN N 128", 128, 128, 2100, 1, 1024, 1, 1, 1, 1, 1.0, 0.0, 0, 0, 0, 0),
    ("split-K f32MN M 1 x bf16MN", 1, 128, 3000, 1, 1024, 0, 1, 1, 1, 1.0, 0.0, 0, 0, 0, 0),
    ("split-K f32MN x f32MN, N 16", 64, 16, 3000, 1, 1024, 0, 1, 0, 1, 1.0, 0.0, 0, 0, 0, 0),
    ("padded f32K x f32MN, K 40, alpha -0.5", 333, 64, 40, 1, 0, 0, 0, 0, 1, -0.5, 0.0, 0, 0, 0, 8),
    ("padded bf16K x bf16K, K 200, batch 3", 300, 128, 200, 3, 0, 1, 0, 1, 0, 1.0, 0.5, 1, 0, 0, 8),
    ("bf16MN x bf16MN, K 72, batch 2", 200, 64, 72, 2, 0, 1, 1, 1, 1, 1.0, 0.0, 0, 0, 0, 0),
]


@pytest.fixture(scope="module")
def net():
    from paper_2501_06377_gb300.surrogate import Surrogate
    n = Surrogate(channels=64, modes=48, blocks=1, max_batch=1, seed=0)
    yield n
    n.close()


def _operand(rows, K, nb, mn, bf, pad, gen):
    """Device operand (FP32 or BF16), its leading dimension and batch stride,
    and its FP64 values after rounding to BF16, as [nb][rows][K]."""
    import torch
    ld = (rows if mn else K) + pad
    per = (K if mn else rows) * ld
    raw = torch.empty(nb * per).uniform_(-1.0, 1.0, generator=gen)
    dev = raw.to(torch.bfloat16).cuda() if bf else raw.cuda()
    r64 = raw.to(torch.bfloat16).double().view(nb, K if mn else rows, ld)
    vals = r64[:, :, :rows].transpose(1, 2) if mn else r64[:, :, :K]
    return dev, ld, (per if nb > 1 else 0), vals.contiguous()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_tensor_core_gemm_matches_fp64_product(net, case):
    import torch
    (_, M, N, K, batch, kchunk, abf, amn, bbf, bmn, alpha, beta, with_bias, ash, bsh, pad) = case
    gen = torch.Generator().manual_seed(zlib.crc32(case[0].encode()))
    split = kchunk > 0
    nz = (K + kchunk - 1) // kchunk if split else batch
    nba = 1 if (split or ash) else batch
    nbb = 1 if (split or bsh) else batch
    A, lda, sA, Av = _operand(M, K, nba, amn, abf, pad, gen)
    B, ldb, sB, Bv = _operand(N, K, nbb, bmn, bbf, pad, gen)
    ldc = N + (4 if pad else 0)
    C0 = torch.empty(nz, M, ldc).uniform_(-1.0, 1.0, generator=gen)
    bias = torch.empty(N).uniform_(-1.0, 1.0, generator=gen)
    Cd = C0.clone().cuda()
    net.debug_gemm(M, N, K, A, amn, lda, sA, B, bmn, ldb, sB, Cd, ldc, M * ldc, alpha=alpha, beta=beta,
                   bias=bias.cuda() if with_bias else None, kchunk=kchunk, batch=nz)
    out = Cd.cpu().double()
    for z in range(nz):
        a = Av[0 if nba == 1 else z]
        b = Bv[0 if nbb == 1 else z]
        k0, k1 = (z * kchunk, min(K, (z + 1) * kchunk)) if split else (0, K)
        a, b = a[:, k0:k1], b[:, k0:k1]
        ref = alpha * (a @ b.T) + beta * C0[z, :, :N].double()
        scale = abs(alpha) * (a.abs() @ b.abs().T) + abs(beta) * C0[z, :, :N].double().abs()
        if with_bias:
            ref = ref + bias.double()[None, :]
            scale = scale + bias.double().abs()[None, :]
        err = (out[z, :, :N] - ref).abs()
        assert bool((err <= 2.4e-7 * (k1 - k0 + 4) * scale + 1e-30).all()), \
            "max err / scale %.3e" % float((err / (scale + 1e-30)).max())
        if pad:  # the padding columns of C are untouched
            assert torch.equal(out[z, :, N:], C0[z, :, N:].double())


def test_bf16_operand_that_tma_cannot_address_is_rejected(net):
    import torch
    from paper_2501_06377_gb300.sft import SFTError, SFT_ERR_ARG
    A = torch.zeros(64 * 41, dtype=torch.bfloat16, device="cuda")  # ld 41: 82-byte rows
    B = torch.zeros(64 * 40, device="cuda")
    Cm = torch.zeros(64 * 64, device="cuda")
    with pytest.raises(SFTError) as e:
        net.debug_gemm(64, 64, 40, A, 0, 41, 0, B, 1, 64, 0, Cm, 64, 0)
    assert e.value.status == SFT_ERR_ARG
