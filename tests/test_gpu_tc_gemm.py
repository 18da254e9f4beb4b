"""The grouped tcgen05 BF16/FP16 GEMM alone, against torch references of the same
product (through the C ABI test hook in include/submat_debug.h)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__ as g
    g.build()
    from paper_2004_10811_gb300 import submat
    return submat


def rand_bf16(count, ld, n, seed, sym=False, scale=1.0):
    import torch
    g = torch.Generator().manual_seed(seed)
    x = torch.zeros(count, ld, ld, dtype=torch.float64)
    x[:, :n, :n] = torch.randn(count, n, n, generator=g, dtype=torch.float64) * scale
    if sym:
        x = 0.5 * (x + x.transpose(1, 2))
    hi = x.to(torch.bfloat16)
    lo = (x - hi.double()).to(torch.bfloat16)
    return x, hi.cuda(), lo.cuda()


@pytest.mark.parametrize("tile_n", [128, 256])
def test_single_tile_plain(sm, tile_n):
    _x, a, _ = rand_bf16(1, 256, 256, 1)
    _y, b, _ = rand_bf16(1, 256, 256, 2)
    c, st = sm.debug_tc_gemm(a, b, tile_n=tile_n)
    ref = a.double() @ b.double().transpose(1, 2)
    err = (c.double() - ref).abs().max().item()
    assert st == "OK" and err < 1e-3 * ref.abs().max().item(), err


@pytest.mark.parametrize("tile_n", [128, 256])
@pytest.mark.parametrize("count,ld,n", [(3, 320, 300), (2, 640, 577), (5, 64, 40)])
def test_ragged_batches_plain(sm, count, ld, n, tile_n):
    _x, a, _ = rand_bf16(count, ld, n, 3)
    _y, b, _ = rand_bf16(count, ld, n, 4)
    c, _ = sm.debug_tc_gemm(a, b, tile_n=tile_n)
    ref = a.double() @ b.double().transpose(1, 2)
    assert (c.double() - ref).abs().max().item() < 2e-3 * ref.abs().max().item()
    assert c[:, n:, :].abs().max().item() == 0.0 and c[:, :, n:].abs().max().item() == 0.0


@pytest.mark.parametrize("tile_n", [128, 256])
def test_split_product_carries_16_bits(sm, tile_n):
    x, ah, al = rand_bf16(2, 384, 350, 5)
    y, bh, bl = rand_bf16(2, 384, 350, 6)
    c, _ = sm.debug_tc_gemm(ah, bh, al, bl, tile_n=tile_n)
    ref = (x @ y.transpose(1, 2)).cuda()
    rel = (c.double() - ref).abs().max().item() / ref.abs().max().item()
    plain, _ = sm.debug_tc_gemm(ah, bh)
    rel_plain = (plain.double() - ref).abs().max().item() / ref.abs().max().item()
    assert rel < 2e-5 and rel < rel_plain / 20, (rel, rel_plain)


@pytest.mark.parametrize("tile_n", [128, 256])
def test_fp16_split_product_carries_19_bits(sm, tile_n):
    """FP16 operands (the Newton-Schulz format): the three-term split keeps
    ~19 bits.  Entries of size 0.05 put most lo parts below FP16's normal
    range (2^-14), so the bound also shows that the tensor cores keep
    subnormal inputs: flushing them would cost ~1e-4 relative."""
    import torch
    g = torch.Generator().manual_seed(11)
    x = torch.zeros(2, 384, 384, dtype=torch.float64)
    y = torch.zeros_like(x)
    x[:, :350, :350] = torch.randn(2, 350, 350, generator=g, dtype=torch.float64) * 0.05
    y[:, :350, :350] = torch.randn(2, 350, 350, generator=g, dtype=torch.float64) * 0.05
    split = lambda t: (t.to(torch.float16), (t - t.to(torch.float16).double()).to(torch.float16))
    (ah, al), (bh, bl) = split(x), split(y)
    assert (al.abs() < 2.0 ** -14).float().mean().item() > 0.5  # mostly subnormal lo parts
    c, st = sm.debug_tc_gemm(ah.cuda(), bh.cuda(), al.cuda(), bl.cuda(), tile_n=tile_n)
    ref = (x @ y.transpose(1, 2)).cuda()
    rel = (c.double() - ref).abs().max().item() / ref.abs().max().item()
    # ~2^-19: the tensor cores' FP32 accumulation, not the operands, limits it
    assert st == "OK" and rel < 4e-6, rel
    # the same product from BF16 pairs is less accurate (measured 2.4x)
    xbh, xbl = x.to(torch.bfloat16), (x - x.to(torch.bfloat16).double()).to(torch.bfloat16)
    ybh, ybl = y.to(torch.bfloat16), (y - y.to(torch.bfloat16).double()).to(torch.bfloat16)
    cb, _ = sm.debug_tc_gemm(xbh.cuda(), ybh.cuda(), xbl.cuda(), ybl.cuda(), tile_n=tile_n)
    rel_b = (cb.double() - ref).abs().max().item() / ref.abs().max().item()
    assert rel < rel_b / 2, (rel, rel_b)


@pytest.mark.parametrize("tile_n", [128, 256])
def test_symmetric_mirror_and_residual(sm, tile_n):
    import torch
    x, xh, xl = rand_bf16(3, 448, 430, 7, sym=True, scale=0.05)
    res = torch.zeros(3, dtype=torch.float64, device="cuda")
    full, _ = sm.debug_tc_gemm(xh, xh, xl, xl, tile_n=tile_n)
    half, _ = sm.debug_tc_gemm(xh, xh, xl, xl, n=430, sym=True, res2=res, tile_n=tile_n)
    assert torch.equal(half, half.transpose(1, 2))
    up = torch.triu(torch.ones(448, 448, dtype=torch.bool, device="cuda"))
    # upper tiles are computed the same way in both launches
    assert (half - full)[:, up].abs().max().item() < 1e-6
    eye = torch.zeros(448, 448, dtype=torch.float64, device="cuda")
    eye[:430, :430] = torch.eye(430, dtype=torch.float64, device="cuda")
    want = ((half.double() - eye) ** 2).sum(dim=(1, 2))
    # the residual is a convergence monitor, summed in FP32 per 32-entry segment
    assert torch.allclose(res, want, rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("tile_n", [128, 256])
def test_bounded_wait_reports_timeout_and_context_survives(sm, tile_n):
    _x, a, _ = rand_bf16(1, 768, 768, 8)
    c, st = sm.debug_tc_gemm(a, a, skip_arrive=True, timeout_s=0.2, allow_timeout=True, tile_n=tile_n)
    assert st == "TIMEOUT"
    c2, st2 = sm.debug_tc_gemm(a, a, tile_n=tile_n)
    ref = a.double() @ a.double().transpose(1, 2)
    assert st2 == "OK" and (c2.double() - ref).abs().max().item() < 2e-3 * ref.abs().max().item()
