"""The tensor-core 3x3 convolution (gea_conv3x3) against the oracle's
convolution on the same bfloat16 operands.

The kernel accumulates in FP32 and the oracle in FP64. With K = 9 cin terms
per output, the FP32 sum is within gamma_K = K 2^-24 times the sum of the
absolute terms, S = conv(|x|, |w|, |b|), of the exact value. A bfloat16
output is that sum rounded to nearest, so it is within that bound plus half
a bfloat16 spacing of each of the two rounded values, (|y| + |y_ref|) 2^-8,
of the rounded oracle value; outside cancellations the two agree exactly or
differ by one unit in the last place, and few outputs differ at all.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2303_10499_gb300 import build as B
    B.build()
    from paper_2303_10499_gb300 import gea as G
    return torch, G


def to_bf16(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16)


def bits(torch, t):
    return t.contiguous().view(torch.int16).cuda()


@pytest.mark.parametrize("cin", [16, 32, 64])
@pytest.mark.parametrize("cout", [16, 32, 64])
@pytest.mark.parametrize("mode", [0, 1, 2], ids=["plain", "pool", "upadd"])
def test_conv3x3_matches_oracle(env, oracle_mod, cin, cout, mode):
    torch, G = env
    from oracle import unet
    rng = np.random.default_rng(1000 * cin + 10 * cout + mode)
    n, h, w = 2, 6, 300          # 300 = 2 x 128 + 44: a ragged last tile
    if mode == 1:
        xs = rng.standard_normal((n, 2 * h, 2 * w, cin))
    else:
        xs = rng.standard_normal((n, h, w, cin))
    x1 = rng.standard_normal((n, h // 2, w // 2, cin)) if mode == 2 else None
    wt = rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin)
    b = rng.standard_normal(cout) * 0.1
    xs, wt = unet.bf16_round(xs), unet.bf16_round(wt)
    x1 = unet.bf16_round(x1) if x1 is not None else None
    if mode == 0:
        xin = xs
    elif mode == 1:
        xin = unet.bf16_round(unet.pool(xs))
    else:
        xin = unet.bf16_round(xs + unet.up(x1))
    ref = unet.conv(xin, wt, b)
    acc = 9 * cin * 2.0 ** -24 * unet.conv(np.abs(xin), np.abs(wt), np.abs(b))
    dx0 = bits(torch, to_bf16(torch, xs))
    dx1 = bits(torch, to_bf16(torch, x1)) if x1 is not None else None
    dw = bits(torch, to_bf16(torch, wt))
    db = torch.tensor(b, dtype=torch.float32).cuda()
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for flags in (0, 1, 2, 3):
        r = np.maximum(ref, 0.0) if flags & 1 else ref
        if flags & 2:
            y = torch.zeros((n, h, w, cout), dtype=torch.float32, device="cuda")
        else:
            y = torch.zeros((n, h, w, cout), dtype=torch.int16, device="cuda")
        G.conv3x3(dx0, dw, y, n, h, w, cin, cout, mode=mode, flags=flags, x1=dx1, bias=db,
                  status=status)
        torch.cuda.synchronize()
        if flags & 2:
            got = y.cpu().numpy().astype(np.float64)
            bad = np.abs(got - r) > acc + 1e-30
            assert not bad.any(), (flags, int(bad.sum()), float(np.abs(got - r).max()))
        else:
            got = y.cpu().view(torch.bfloat16).float().numpy().astype(np.float64)
            want = unet.bf16_round(r)
            diff = np.abs(got - want)
            bad = diff > acc + (np.abs(got) + np.abs(want)) * 2.0 ** -8
            assert not bad.any(), (flags, int(bad.sum()), float(diff.max()))
            # boundary cases only
            assert (diff > 0).mean() < 1e-3, (flags, float((diff > 0).mean()))
    assert int(status.item()) == 0


@pytest.mark.parametrize("cin,cout,mode,n,h", [(16, 16, 0, 1, 1700), (16, 16, 1, 1, 1700),
                                                (32, 64, 2, 1, 900), (64, 32, 0, 2, 300),
                                                (64, 64, 0, 2, 300), (64, 64, 2, 2, 300)])
def test_conv3x3_column_runs(env, oracle_mod, cin, cout, mode, n, h):
    """Images tall enough that every CTA walks several tiles down a tile
    column (the ring of staged rows, the row prefetched during the previous
    tile's MMA batch, the two accumulator buffers), with ranges that cross
    from one column or image into the next."""
    torch, G = env
    from oracle import unet
    rng = np.random.default_rng(7 * cin + 3 * cout + mode + h)
    w = 260                      # 2 x 128 + 4: a ragged last tile column
    xs = rng.standard_normal((n, 2 * h, 2 * w, cin) if mode == 1 else (n, h, w, cin))
    x1 = rng.standard_normal((n, h // 2, w // 2, cin)) if mode == 2 else None
    wt = rng.standard_normal((cout, 3, 3, cin)) / np.sqrt(9 * cin)
    b = rng.standard_normal(cout) * 0.1
    xs, wt = unet.bf16_round(xs), unet.bf16_round(wt)
    x1 = unet.bf16_round(x1) if x1 is not None else None
    xin = xs if mode == 0 else (unet.bf16_round(unet.pool(xs)) if mode == 1 else unet.bf16_round(xs + unet.up(x1)))
    ref = unet.conv(xin, wt, b)
    acc = 9 * cin * 2.0 ** -24 * unet.conv(np.abs(xin), np.abs(wt), np.abs(b))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    y = torch.zeros((n, h, w, cout), dtype=torch.float32, device="cuda")
    G.conv3x3(bits(torch, to_bf16(torch, xs)), bits(torch, to_bf16(torch, wt)), y, n, h, w, cin, cout,
              mode=mode, flags=2, x1=bits(torch, to_bf16(torch, x1)) if x1 is not None else None,
              bias=torch.tensor(b, dtype=torch.float32).cuda(), status=status)
    torch.cuda.synchronize()
    got = y.cpu().numpy().astype(np.float64)
    bad = np.abs(got - ref) > acc + 1e-30
    assert not bad.any(), (int(bad.sum()), float(np.abs(got - ref).max()))
    assert int(status.item()) == 0


def test_conv3x3_rejects_bad_arguments(env):
    torch, G = env
    x = torch.zeros(16, dtype=torch.int16, device="cuda")
    for kw in (dict(cin=8, cout=16), dict(cin=16, cout=48), dict(cin=16, cout=16, mode=3)):
        with pytest.raises(G.GeaError):
            G.conv3x3(x, x, x, 1, 4, 4, kw["cin"], kw["cout"], mode=kw.get("mode", 0))
    with pytest.raises(G.GeaError):   # UPADD needs even sizes and x1
        G.conv3x3(x, x, x, 1, 3, 4, 16, 16, mode=2, x1=x)
